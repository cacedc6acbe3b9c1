// One cudaMalloc per handle; sub-buffers are carved out with 256-byte alignment.  A sizing pass
// (base == nullptr) only counts bytes, which is what ipeps_footprint_bytes reports.
#pragma once
#include <cstddef>
#include <vector>

namespace ipeps {

struct Arena {
  char* base = nullptr;
  size_t used = 0;
  template <class T>
  T* take(size_t count) {
    size_t off = (used + 255) & ~size_t(255);
    used = off + count * sizeof(T);
    return base ? reinterpret_cast<T*>(base + off) : reinterpret_cast<T*>(off + 256);
  }
};

// Host staging area for device arrays of device pointers (batched GEMM / SVD operands).  Offsets
// are handed out while building; after upload, dev() turns an offset into a device address.
struct PtrPool {
  std::vector<const void*> host;
  void** base = nullptr;
  size_t add(const std::vector<const void*>& v) {
    size_t off = host.size();
    host.insert(host.end(), v.begin(), v.end());
    return off;
  }
  template <class T>
  T dev(size_t off) const { return reinterpret_cast<T>(base + off); }
};

}  // namespace ipeps
