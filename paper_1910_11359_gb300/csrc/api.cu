// C-ABI of libipeps (declarations and documentation in include/ipeps.h, include/ipeps_kernels.h).
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/ipeps.h"
#include "../../include/ipeps_kernels.h"
#include "ctx.cuh"
#include "measure.cuh"
#include "model.cuh"
#include "orth.cuh"
#include "prof.cuh"
#include "tc_gemm.cuh"

using namespace ipeps;

struct ipeps_ctx {
  Ctx c;
  MeasureWork mw;
  MeasureOff moff;
  MeasurePlan mplan;
  std::vector<int> last_sweeps;
  std::vector<double> last_delta;
  std::vector<double> last_eps;
  double t_measured = 0.0;
};

namespace {

ipeps_status fail(ipeps_h h, ipeps_status s, const std::string& msg) {
  if (h) h->c.msg = msg;
  set_thread_error(msg);
  return s;
}

ipeps_status from_rc(ipeps_h h, int rc) {
  if (rc == 0) return IPEPS_OK;
  std::string m = thread_error_message();
  if (h) h->c.msg = m;
  return (ipeps_status)rc;
}

// device error word -> status (and reset)
ipeps_status check_dev(ipeps_h h) {
  unsigned e = 0;
  cudaError_t ce = cudaMemcpyAsync(&e, h->c.derr, sizeof(unsigned), cudaMemcpyDeviceToHost, h->c.st);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(h->c.st);
  if (ce != cudaSuccess) return from_rc(h, cuda_fail(ce, "sync", __FILE__, __LINE__));
  if (e) {
    cudaMemsetAsync(h->c.derr, 0, sizeof(unsigned), h->c.st);
    if (e & DEV_NONFINITE) return fail(h, IPEPS_ENAN, "non-finite value in a device kernel");
    if (e & DEV_JACOBI_CAP) return fail(h, IPEPS_ENOCONV, "Jacobi SVD hit its sweep limit");
    if (e & DEV_BAD_SIZE) return fail(h, IPEPS_EINVAL, "device kernel rejected a size");
    if (e & DEV_TIMEOUT) return fail(h, IPEPS_ETIMEOUT, "a bounded device-side wait ran out");
  }
  return IPEPS_OK;
}

ipeps_status validate(const ipeps_params* p, std::string* why) {
  if (!p) { *why = "params is NULL"; return IPEPS_EINVAL; }
  if (p->batch < 1 || p->batch > 4096) { *why = "batch must be in [1, 4096]"; return IPEPS_EINVAL; }
  if (p->d_A < 2 || p->d_A > 5) { *why = "d_A must be in [2, 5]"; return IPEPS_EINVAL; }
  if (p->D < 2 || p->D > 8) { *why = "D must be in [2, 8]"; return IPEPS_EINVAL; }
  if (p->D * p->D < 2 * p->d_A) {
    *why = "the reduced simple update needs D^2 >= d = 2 d_A";
    return IPEPS_EUNSUPPORTED;
  }
  {
    const int d = 2 * p->d_A, nt = d * d * p->D;
    if (!jacobi_svd_supported(nt, nt) || !jacobi_svd_fits(p->D * p->D * p->D, d * p->D)) {
      *why = "d^2 D too large for the simple-update SVD";
      return IPEPS_EUNSUPPORTED;
    }
  }
  if (p->chi < p->D * p->D) { *why = "chi must be >= D^2"; return IPEPS_EINVAL; }
  if (p->chi > 2048) { *why = "chi above 2048 is not supported"; return IPEPS_EUNSUPPORTED; }
  if (p->trotter_order != 1 && p->trotter_order != 2) { *why = "trotter_order must be 1 or 2"; return IPEPS_EINVAL; }
  if (!(p->dt > 0.0)) { *why = "dt must be > 0"; return IPEPS_EINVAL; }
  if (p->precision != IPEPS_FP64 && p->precision != IPEPS_SPLIT_BF16X3 && p->precision != IPEPS_SPLIT_TF32X3) {
    *why = "precision must be IPEPS_FP64, IPEPS_SPLIT_BF16X3 or IPEPS_SPLIT_TF32X3";
    return IPEPS_EINVAL;
  }
  if (!p->J || !p->V || !p->h) { *why = "J, V, h arrays are required"; return IPEPS_EINVAL; }
  const int N = p->chi * p->D * p->D;
  const int k = subspace_size(p->chi, N);
  const bool sub = p->projector_svd == 2 ? k < N : (p->projector_svd == 1 ? false : N > 2 * k);
  if (p->projector_svd < 0 || p->projector_svd > 2) { *why = "projector_svd must be 0, 1 or 2"; return IPEPS_EINVAL; }
  if (sub && k > 256) { *why = "the projector subspace (chi + max(8, chi / 4)) must not exceed 256"; return IPEPS_EUNSUPPORTED; }
  if (sub ? !jacobi_svd_supported(N, k) : !jacobi_svd_fits(N, N)) {
    *why = "chi * D^2 too large for the projector SVD";
    return IPEPS_EUNSUPPORTED;
  }
  return IPEPS_OK;
}

void carve_all(ipeps_ctx* x) {
  Ctx& c = x->c;
  Arena& a = c.arena;
  const int B = c.B, d = c.d, D = c.D;
  const long long D4 = (long long)D * D * D * D, D3 = (long long)D * D * D;
  const int n = d * D, nt = n * d;
  c.GA = a.take<cplx>((size_t)B * d * D4);
  c.GB = a.take<cplx>((size_t)B * d * D4);
  c.lam = a.take<double>((size_t)B * 4 * D);
  c.eps = a.take<double>(B);
  c.dJ = a.take<double>(B); c.dV = a.take<double>(B); c.dh = a.take<double>(B);
  c.ddelta = a.take<double>(2);
  c.gates = a.take<cplx>((size_t)2 * B * d * d * d * d);
  c.bondop = a.take<cplx>((size_t)B * d * d * d * d);
  c.derr = a.take<unsigned>(1);
  c.dflag = a.take<int>(1);
  c.loopctl = a.take<int>(4);
  SuWork& s = c.su;
  s.Amat = a.take<cplx>((size_t)B * D3 * n); s.Bmat = a.take<cplx>((size_t)B * D3 * n);
  s.UA = a.take<cplx>((size_t)B * D3 * n); s.UB = a.take<cplx>((size_t)B * D3 * n);
  s.SA = a.take<double>((size_t)B * n); s.SB = a.take<double>((size_t)B * n);
  s.VA = a.take<cplx>((size_t)B * n * n); s.VB = a.take<cplx>((size_t)B * n * n);
  s.theta = a.take<cplx>((size_t)B * nt * nt);
  s.X = a.take<cplx>((size_t)B * nt * nt); s.Y = a.take<cplx>((size_t)B * nt * nt);
  s.Stheta = a.take<double>((size_t)B * nt);
  s.kept = a.take<int>(B);
  s.tgwork = nullptr;
  s.tgwork_bytes = 0;
  if (!jacobi_svd_fits(nt, nt)) {
    s.tgwork_bytes = jacobi_svd_global_bytes(nt, nt, B);
    s.tgwork = a.take<cplx>(s.tgwork_bytes / sizeof(cplx) + 1);
  }
  ctm_carve(c);
  measure_carve(a, x->mw, B, d, D, c.chi);
}

struct SuOff { size_t qA, qU, qS, qV, tA, tU, tS, tV; };

SuOff su_build(Ctx& c) {
  const int B = c.B, d = c.d, D = c.D;
  const long long D3 = (long long)D * D * D;
  const int n = d * D, nt = n * d;
  SuWork& s = c.su;
  std::vector<const void*> qA, qU, qS, qV, tA, tU, tS, tV;
  for (int side = 0; side < 2; ++side)
    for (int b = 0; b < B; ++b) {
      qA.push_back((side ? s.Bmat : s.Amat) + (size_t)b * D3 * n);
      qU.push_back((side ? s.UB : s.UA) + (size_t)b * D3 * n);
      qS.push_back((side ? s.SB : s.SA) + (size_t)b * n);
      qV.push_back((side ? s.VB : s.VA) + (size_t)b * n * n);
    }
  for (int b = 0; b < B; ++b) {
    tA.push_back(s.theta + (size_t)b * nt * nt);
    tU.push_back(s.X + (size_t)b * nt * nt);
    tS.push_back(s.Stheta + (size_t)b * nt);
    tV.push_back(s.Y + (size_t)b * nt * nt);
  }
  SuOff o;
  o.qA = c.pool.add(qA); o.qU = c.pool.add(qU); o.qS = c.pool.add(qS); o.qV = c.pool.add(qV);
  o.tA = c.pool.add(tA); o.tU = c.pool.add(tU); o.tS = c.pool.add(tS); o.tV = c.pool.add(tV);
  return o;
}

void su_resolve(Ctx& c, const SuOff& o) {
  SuWork& s = c.su;
  s.qA = c.pool.dev<const cplx* const*>(o.qA); s.qU = c.pool.dev<cplx* const*>(o.qU);
  s.qS = c.pool.dev<double* const*>(o.qS); s.qV = c.pool.dev<cplx* const*>(o.qV);
  s.tA = c.pool.dev<const cplx* const*>(o.tA); s.tU = c.pool.dev<cplx* const*>(o.tU);
  s.tS = c.pool.dev<double* const*>(o.tS); s.tV = c.pool.dev<cplx* const*>(o.tV);
}

void set_params(Ctx& c, const ipeps_params* p) {
  c.B = p->batch; c.dA = p->d_A; c.d = 2 * p->d_A; c.D = p->D; c.D2 = p->D * p->D; c.chi = p->chi;
  c.N = c.chi * c.D2; c.order = p->trotter_order; c.dt = p->dt; c.precision = p->precision;
  c.seed = p->seed;
  c.cut_rel = p->ctm_cut_rel > 0.0 ? p->ctm_cut_rel : 1e-10;
  c.k = subspace_size(c.chi, c.N);
  c.subspace = p->projector_svd == 2 ? c.k < c.N : (p->projector_svd == 1 ? false : c.N > 2 * c.k);
}

}  // namespace

extern "C" {

ipeps_status ipeps_footprint_bytes(const ipeps_params* p, size_t* bytes) {
  std::string why;
  if (!bytes) return fail(nullptr, IPEPS_EINVAL, "bytes is NULL");
  ipeps_status s = validate(p, &why);
  if (s != IPEPS_OK) return fail(nullptr, s, why);
  ipeps_ctx tmp;
  set_params(tmp.c, p);
  carve_all(&tmp);
  *bytes = tmp.c.arena.used;
  return IPEPS_OK;
}

ipeps_status ipeps_init(const ipeps_params* p, void* cuda_stream, ipeps_h* out) {
  std::string why;
  if (!out) return fail(nullptr, IPEPS_EINVAL, "out is NULL");
  *out = nullptr;
  ipeps_status s = validate(p, &why);
  if (s != IPEPS_OK) return fail(nullptr, s, why);
  ipeps_ctx* x = new (std::nothrow) ipeps_ctx();
  if (!x) return fail(nullptr, IPEPS_ENOMEM, "host allocation failed");
  Ctx& c = x->c;
  set_params(c, p);
  c.st = (cudaStream_t)cuda_stream;
  c.J.assign(p->J, p->J + c.B); c.V.assign(p->V, p->V + c.B); c.h.assign(p->h, p->h + c.B);
  // sizing pass, one allocation, carving pass
  carve_all(x);
  size_t bytes = c.arena.used;
  c.arena = Arena();
  if (cudaMalloc(&c.dev_base, bytes) != cudaSuccess) {
    cudaGetLastError();
    delete x;
    return fail(nullptr, IPEPS_ENOMEM, "cudaMalloc of the device arena failed");
  }
  c.arena.base = (char*)c.dev_base;
  carve_all(x);
  // device pointer arrays
  SuOff so = su_build(c);
  ctm_build_plans(c);
  measure_build(c, x->mw, c.pool, x->moff);
  const size_t pbytes = c.pool.host.size() * sizeof(void*);
  if (cudaMalloc(&c.dev_ptrs, pbytes) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(c.dev_base);
    delete x;
    return fail(nullptr, IPEPS_ENOMEM, "cudaMalloc of the pointer tables failed");
  }
  c.pool.base = (void**)c.dev_ptrs;
  if (cudaHostAlloc((void**)&c.hflag, 4 * sizeof(int), cudaHostAllocDefault) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(c.dev_ptrs);
    cudaFree(c.dev_base);
    delete x;
    return fail(nullptr, IPEPS_ENOMEM, "cudaHostAlloc of the convergence flag failed");
  }
  ipeps_h h = x;
  auto cuda = [&](cudaError_t e, const char* what) -> ipeps_status {
    if (e == cudaSuccess) return IPEPS_OK;
    return from_rc(h, cuda_fail(e, what, __FILE__, __LINE__));
  };
  if ((s = cuda(cudaMemcpy(c.dev_ptrs, c.pool.host.data(), pbytes, cudaMemcpyHostToDevice), "pointer tables"))) goto bad;
  su_resolve(c, so);
  ctm_resolve_plans(c);
  measure_resolve(c.pool, x->moff, x->mplan);
  {
    // Trotter sequence: bonds named by A's leg (u=0, l=1, d=2, r=3)
    double deltas[2];
    if (c.order == 1) {
      c.ndelta = 1; deltas[0] = c.dt; deltas[1] = 0.0;
      c.seq = {{3, 0}, {0, 0}, {1, 0}, {2, 0}};
    } else {
      c.ndelta = 2; deltas[0] = 0.5 * c.dt; deltas[1] = c.dt;
      c.seq = {{3, 0}, {0, 0}, {1, 0}, {2, 1}, {1, 0}, {0, 0}, {3, 0}};
    }
    if ((s = cuda(cudaMemcpyAsync(c.ddelta, deltas, sizeof(deltas), cudaMemcpyHostToDevice, c.st), "deltas"))) goto bad;
    if ((s = cuda(cudaMemcpyAsync(c.dJ, c.J.data(), sizeof(double) * c.B, cudaMemcpyHostToDevice, c.st), "J"))) goto bad;
    if ((s = cuda(cudaMemcpyAsync(c.dV, c.V.data(), sizeof(double) * c.B, cudaMemcpyHostToDevice, c.st), "V"))) goto bad;
    if ((s = cuda(cudaMemcpyAsync(c.dh, c.h.data(), sizeof(double) * c.B, cudaMemcpyHostToDevice, c.st), "h"))) goto bad;
    if ((s = cuda(cudaMemsetAsync(c.eps, 0, sizeof(double) * c.B, c.st), "eps"))) goto bad;
    if ((s = cuda(cudaMemsetAsync(c.derr, 0, sizeof(unsigned), c.st), "err"))) goto bad;
    if ((s = from_rc(h, build_gates(c.dJ, c.dV, c.dh, c.ddelta, c.ndelta, c.B, c.d, c.dA, c.gates, c.st)))) goto bad;
    if ((s = from_rc(h, build_bond_ops(c.dJ, c.dV, c.B, c.d, c.dA, c.bondop, c.st)))) goto bad;
    if ((s = from_rc(h, init_state(c.GA, c.GB, c.lam, c.d, c.dA, c.D, c.B, c.st)))) goto bad;
    if ((s = cuda(cudaStreamSynchronize(c.st), "init sync"))) goto bad;
  }
  x->last_sweeps.assign(c.B, 0);
  x->last_delta.assign(c.B, 0.0);
  x->last_eps.assign(c.B, 0.0);
  *out = h;
  return IPEPS_OK;
bad:
  cudaFreeHost(c.hflag);
  cudaFree(c.dev_ptrs);
  cudaFree(c.dev_base);
  delete x;
  return s;
}

ipeps_status ipeps_destroy(ipeps_h h) {
  if (!h) return IPEPS_OK;
  cudaStreamSynchronize(h->c.st);
  if (h->c.conv_exec) cudaGraphExecDestroy(h->c.conv_exec);
  if (h->c.cap_st) cudaStreamDestroy(h->c.cap_st);
  cudaFreeHost(h->c.hflag);
  cudaFree(h->c.dev_ptrs);
  cudaFree(h->c.dev_base);
  delete h;
  return IPEPS_OK;
}

ipeps_status ipeps_set_graphs(ipeps_h h, int enable) {
  if (!h) return fail(h, IPEPS_EINVAL, "NULL handle");
  h->c.graphs = enable != 0;
  return IPEPS_OK;
}

const char* ipeps_last_error(ipeps_h h) { return h ? h->c.msg.c_str() : thread_error_message(); }

ipeps_status ipeps_set_tensors(ipeps_h h, const double* gA, const double* gB, const double* lambda) {
  if (!h || !gA || !gB) return fail(h, IPEPS_EINVAL, "NULL argument");
  Ctx& c = h->c;
  const size_t ng = (size_t)c.B * c.d * c.D2 * c.D2;
  std::vector<double> lam((size_t)c.B * 4 * c.D, 1.0);
  if (lambda) lam.assign(lambda, lambda + lam.size());
  if (cudaMemcpyAsync(c.GA, gA, ng * sizeof(cplx), cudaMemcpyHostToDevice, c.st) != cudaSuccess ||
      cudaMemcpyAsync(c.GB, gB, ng * sizeof(cplx), cudaMemcpyHostToDevice, c.st) != cudaSuccess ||
      cudaMemcpyAsync(c.lam, lam.data(), lam.size() * sizeof(double), cudaMemcpyHostToDevice, c.st) != cudaSuccess ||
      cudaStreamSynchronize(c.st) != cudaSuccess)
    return from_rc(h, cuda_fail(cudaGetLastError(), "set_tensors", __FILE__, __LINE__));
  return IPEPS_OK;
}

ipeps_status ipeps_trotter_step(ipeps_h h, int n_steps, double* trunc_err_out) {
  if (!h || n_steps < 0) return fail(h, IPEPS_EINVAL, "bad handle or n_steps");
  Ctx& c = h->c;
  const long long gstride = (long long)c.B * c.d * c.d * c.d * c.d;
  for (int step = 0; step < n_steps; ++step)
    for (auto& lg : c.seq) {
      int rc = su_bond_update(c.su, c.GA, c.GB, c.lam, c.eps, c.gates + (size_t)lg.second * gstride,
                              lg.first, c.d, c.D, c.B, c.derr, c.st);
      if (rc) return from_rc(h, rc);
    }
  c.t += n_steps * c.dt;
  if (trunc_err_out) {
    if (cudaMemcpyAsync(trunc_err_out, c.eps, sizeof(double) * c.B, cudaMemcpyDeviceToHost, c.st) != cudaSuccess)
      return from_rc(h, cuda_fail(cudaGetLastError(), "eps copy", __FILE__, __LINE__));
    ipeps_status s = check_dev(h);
    if (s != IPEPS_OK) return s;
  }
  return IPEPS_OK;
}

ipeps_status ctmrg_reset(ipeps_h h) {
  if (!h) return fail(h, IPEPS_EINVAL, "NULL handle");
  h->c.env_valid = false;
  return IPEPS_OK;
}

// End of a sweep inside the convergence graph: counts it and continues while fewer than the limit
// ran and (with a tolerance) some instance is still open.
__global__ void conv_test_kernel(const int* frozen, int B, int* ctl, int use_tol, cudaGraphConditionalHandle h) {
  __shared__ int open;
  if (threadIdx.x == 0) open = 0;
  __syncthreads();
  for (int b = threadIdx.x; b < B; b += blockDim.x)
    if (!frozen[b]) open = 1;
  __syncthreads();
  if (threadIdx.x == 0) {
    const int s = ctl[0] + 1;
    ctl[0] = s;
    loop_set(h, 1, s < ctl[1] && (!use_tol || open));
  }
}

// Captures the convergence loop (sweep, corner spectra, test) as one graph: a WHILE node over
// sweeps whose body holds one WHILE node per projector's subspace rounds.
static int capture_converge(Ctx& c, double tol_eff, bool use_tol) {
  if (!c.cap_st) IPEPS_CUDA_TRY(cudaStreamCreateWithFlags(&c.cap_st, cudaStreamNonBlocking));
  GraphBuilder gb;
  cudaGraphExec_t exec = nullptr;
  // the routines below issue their work on c.st: point it at the capture stream meanwhile (nothing
  // runs during a capture; the graph is launched on the handle's own stream)
  const cudaStream_t user_st = c.st;
  c.st = c.cap_st;
  int rc = gb.begin(c.st);
  cudaGraphConditionalHandle hs = 0;
  c.gb = &gb;
  if (!rc) rc = gb.loop_begin(c.loopctl, &hs);
  if (!rc) rc = ctm_sweep(c);
  if (!rc) rc = ctm_spectra(c, tol_eff, 0);
  if (!rc) {
    conv_test_kernel<<<1, 128, 0, c.st>>>(c.w.frozen, c.B, c.loopctl, use_tol ? 1 : 0, hs);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) rc = cuda_fail(e, "conv test launch", __FILE__, __LINE__);
  }
  if (!rc) rc = gb.loop_end();
  if (!rc) rc = gb.end(&exec);
  c.gb = nullptr;
  c.st = user_st;
  if (rc) {
    gb.abandon();
    return rc;
  }
  if (c.conv_exec) cudaGraphExecDestroy(c.conv_exec);
  c.conv_exec = exec;
  c.conv_tol = use_tol ? tol_eff : -1.0;
  return 0;
}

static bool slots_warm(const Ctx& c) {
  for (int f = 0; f < 4; ++f)
    for (int x = 0; x < 2; ++x)
      if (!c.slot_warm[f][x]) return false;
  return true;
}

ipeps_status ctmrg_converge(ipeps_h h, double tol, int max_sweeps, int* sweeps_out, double* delta_out) {
  if (!h || max_sweeps < 1) return fail(h, IPEPS_EINVAL, "bad handle or max_sweeps");
  Ctx& c = h->c;
  const int B = c.B;
  int rc;
  if ((rc = ctm_prepare_tensors(c))) return from_rc(h, rc);
  if (!c.env_valid && (rc = ctm_init_env(c))) return from_rc(h, rc);
  cudaMemsetAsync(c.w.frozen, 0, sizeof(int) * B, c.st);
  cudaMemsetAsync(c.w.sweeps, 0, sizeof(int) * B, c.st);
  if ((rc = ctm_spectra(c, tol, 1))) return from_rc(h, rc);
  std::vector<int> frozen(B, 0);
  // split precision: its contractions leave a noise floor in the corner spectra (near 1e-6 for
  // BF16x3, 1e-8 for TF32x3), so a requested tolerance below split_tol_floor is raised to it (the
  // stall rule covers the rest)
  const double floor_tol = split_tol_floor(c.precision);
  const double tol_eff = tol > 0.0 ? (tol < floor_tol ? floor_tol : tol) : -1.0;
  // Sweeps run eagerly (a host readback of the frozen flags after each) until every projector slot
  // has its warm start; the rest run as one launch of the convergence graph, in which the device
  // decides when to stop.  Both run the same kernels in the same order.
  int s = 0;
  bool all = false;
  const bool graphs = c.graphs && !prof_enabled();
  while (s < max_sweeps && !all && !(graphs && slots_warm(c))) {
    if ((rc = ctm_sweep(c))) return from_rc(h, rc);
    if ((rc = ctm_spectra(c, tol_eff, 0))) return from_rc(h, rc);
    ++s;
    if (tol > 0.0) {
      if (cudaMemcpyAsync(frozen.data(), c.w.frozen, sizeof(int) * B, cudaMemcpyDeviceToHost, c.st) != cudaSuccess)
        return from_rc(h, cuda_fail(cudaGetLastError(), "frozen copy", __FILE__, __LINE__));
      ipeps_status st = check_dev(h);
      if (st != IPEPS_OK && st != IPEPS_ENOCONV) return st;
      all = true;
      for (int b = 0; b < B; ++b) all = all && frozen[b];
    }
  }
  if (s < max_sweeps && !all) {
    const double key = tol > 0.0 ? tol_eff : -1.0;
    if (!c.conv_exec || c.conv_tol != key) {
      if ((rc = capture_converge(c, tol_eff, tol > 0.0))) return from_rc(h, rc);
    }
    c.hflag[1] = max_sweeps - s;
    if (cudaMemcpyAsync(c.loopctl + 1, c.hflag + 1, sizeof(int), cudaMemcpyHostToDevice, c.st) != cudaSuccess ||
        cudaGraphLaunch(c.conv_exec, c.st) != cudaSuccess)
      return from_rc(h, cuda_fail(cudaGetLastError(), "convergence graph launch", __FILE__, __LINE__));
  }
  h->last_sweeps.assign(B, 0);
  h->last_delta.assign(B, 0.0);
  cudaMemcpyAsync(h->last_sweeps.data(), c.w.sweeps, sizeof(int) * B, cudaMemcpyDeviceToHost, c.st);
  cudaMemcpyAsync(h->last_delta.data(), c.w.delta, sizeof(double) * B, cudaMemcpyDeviceToHost, c.st);
  cudaMemcpyAsync(h->last_eps.data(), c.eps, sizeof(double) * B, cudaMemcpyDeviceToHost, c.st);
  cudaMemcpyAsync(frozen.data(), c.w.frozen, sizeof(int) * B, cudaMemcpyDeviceToHost, c.st);
  ipeps_status st = check_dev(h);
  h->t_measured = c.t;
  if (st != IPEPS_OK && st != IPEPS_ENOCONV) return st;
  if (sweeps_out) memcpy(sweeps_out, h->last_sweeps.data(), sizeof(int) * B);
  if (delta_out) memcpy(delta_out, h->last_delta.data(), sizeof(double) * B);
  if (tol > 0.0)
    for (int b = 0; b < B; ++b)
      if (!frozen[b]) return fail(h, IPEPS_ENOCONV, "CTMRG reached max_sweeps without converging");
  return st;
}

ipeps_status ipeps_measure(ipeps_h h, ipeps_obs* out) {
  if (!h || !out) return fail(h, IPEPS_EINVAL, "NULL argument");
  Ctx& c = h->c;
  if (!c.env_valid) return fail(h, IPEPS_EINVAL, "no environment: call ctmrg_converge first");
  std::vector<double> o((size_t)kObsPerInstance * c.B);
  int rc = measure_run(c, h->mw, h->mplan, o.data());
  if (rc) return from_rc(h, rc);
  ipeps_status st = check_dev(h);
  if (st != IPEPS_OK) return st;
  for (int b = 0; b < c.B; ++b) {
    ipeps_obs& r = out[b];
    const double* v = &o[(size_t)b * kObsPerInstance];
    r.t = h->t_measured;
    r.nA = v[0]; r.nB = v[1]; r.imbalance = v[2]; r.tauzA = v[3]; r.tauzB = v[4];
    r.energy = v[5]; r.purityA = v[6];
    r.renyi1A = v[8]; r.renyi_halfA = v[9]; r.renyi2A = v[10];
    r.trunc_err_acc = h->last_eps[b];
    r.ctm_sweeps = h->last_sweeps[b];
    r.ctm_delta = h->last_delta[b];
  }
  return IPEPS_OK;
}

ipeps_status ipeps_corner_spectrum(ipeps_h h, int inst, int pos, int corner, double* sv_out) {
  if (!h || !sv_out) return fail(h, IPEPS_EINVAL, "NULL argument");
  Ctx& c = h->c;
  if (inst < 0 || inst >= c.B || pos < 0 || pos >= NPOS || corner < 0 || corner > 3)
    return fail(h, IPEPS_EINVAL, "index out of range");
  if (!c.env_valid) return fail(h, IPEPS_EINVAL, "no environment");
  SvdDesc sd;
  sd.m = c.chi; sd.n = c.chi; sd.batch = 16 * c.B;
  sd.A = c.w.csA; sd.lda = c.chi; sd.U = nullptr; sd.ldu = 0; sd.S = c.w.csS; sd.V = nullptr; sd.ldv = 0;
  sd.tol = 4e-16 * c.chi; sd.max_sweeps = 80; sd.err = c.derr; sd.sweeps_out = nullptr; sd.skip = nullptr;
  int rc = jacobi_svd(sd, c.st);
  if (rc) return from_rc(h, rc);
  std::vector<double> s(c.chi);
  cudaMemcpyAsync(s.data(), c.w.cs + (size_t)((corner * NPOS + pos) * c.B + inst) * c.chi,
                  sizeof(double) * c.chi, cudaMemcpyDeviceToHost, c.st);
  ipeps_status st = check_dev(h);
  if (st != IPEPS_OK) return st;
  for (int k = 0; k < c.chi; ++k) sv_out[k] = s[0] > 0.0 ? s[k] / s[0] : 0.0;
  return IPEPS_OK;
}

ipeps_status ipeps_get_env(ipeps_h h, int inst, double* C_out, double* T_out) {
  if (!h || !C_out || !T_out) return fail(h, IPEPS_EINVAL, "NULL argument");
  Ctx& c = h->c;
  if (inst < 0 || inst >= c.B) return fail(h, IPEPS_EINVAL, "instance out of range");
  if (!c.env_valid) return fail(h, IPEPS_EINVAL, "no environment: call ctmrg_converge first");
  const size_t nC = (size_t)c.chi * c.chi, nT = (size_t)c.chi * c.D2 * c.chi;
  for (int i = 0; i < 4; ++i)
    for (int p = 0; p < NPOS; ++p) {
      cplx* dC = (cplx*)C_out + (size_t)(i * NPOS + p) * nC;
      cplx* dT = (cplx*)T_out + (size_t)(i * NPOS + p) * nT;
      if (cudaMemcpyAsync(dC, c.Cenv[i][p] + (size_t)inst * nC, nC * sizeof(cplx), cudaMemcpyDeviceToHost,
                          c.st) != cudaSuccess ||
          cudaMemcpyAsync(dT, c.Tenv[i][p] + (size_t)inst * nT, nT * sizeof(cplx), cudaMemcpyDeviceToHost,
                          c.st) != cudaSuccess)
        return from_rc(h, cuda_fail(cudaGetLastError(), "get_env", __FILE__, __LINE__));
    }
  return check_dev(h);
}

ipeps_status ipeps_set_env(ipeps_h h, int inst, const double* C_in, const double* T_in) {
  if (!h || !C_in || !T_in) return fail(h, IPEPS_EINVAL, "NULL argument");
  Ctx& c = h->c;
  if (inst < 0 || inst >= c.B) return fail(h, IPEPS_EINVAL, "instance out of range");
  int rc;
  if (!c.env_valid) {
    // the other instances get the traced start of their current tensors
    if ((rc = ctm_prepare_tensors(c)) || (rc = ctm_init_env(c))) return from_rc(h, rc);
  }
  const size_t nC = (size_t)c.chi * c.chi, nT = (size_t)c.chi * c.D2 * c.chi;
  for (int i = 0; i < 4; ++i)
    for (int p = 0; p < NPOS; ++p) {
      const cplx* sC = (const cplx*)C_in + (size_t)(i * NPOS + p) * nC;
      const cplx* sT = (const cplx*)T_in + (size_t)(i * NPOS + p) * nT;
      if (cudaMemcpyAsync(c.Cenv[i][p] + (size_t)inst * nC, sC, nC * sizeof(cplx), cudaMemcpyHostToDevice,
                          c.st) != cudaSuccess ||
          cudaMemcpyAsync(c.Tenv[i][p] + (size_t)inst * nT, sT, nT * sizeof(cplx), cudaMemcpyHostToDevice,
                          c.st) != cudaSuccess)
        return from_rc(h, cuda_fail(cudaGetLastError(), "set_env", __FILE__, __LINE__));
    }
  return check_dev(h);
}

ipeps_status ipeps_get_lambda(ipeps_h h, double* lambda_out) {
  if (!h || !lambda_out) return fail(h, IPEPS_EINVAL, "NULL argument");
  Ctx& c = h->c;
  cudaMemcpyAsync(lambda_out, c.lam, sizeof(double) * c.B * 4 * c.D, cudaMemcpyDeviceToHost, c.st);
  return check_dev(h);
}

ipeps_status ipeps_get_tensors(ipeps_h h, double* gA, double* gB) {
  if (!h || !gA || !gB) return fail(h, IPEPS_EINVAL, "NULL argument");
  Ctx& c = h->c;
  const size_t ng = (size_t)c.B * c.d * c.D2 * c.D2;
  cudaMemcpyAsync(gA, c.GA, ng * sizeof(cplx), cudaMemcpyDeviceToHost, c.st);
  cudaMemcpyAsync(gB, c.GB, ng * sizeof(cplx), cudaMemcpyDeviceToHost, c.st);
  return check_dev(h);
}

// ----------------------------------------------------------------------------- kernel test hooks
int ipeps_kernel_zgemm(int M, int N, int K, int batch, int opA, int opB, const double* A, long long lda,
                       long long sA, const double* B, long long ldb, long long sB, double* C,
                       long long ldc, long long sC, void* stream) {
  GemmDesc g;
  memset(&g, 0, sizeof(g));
  g.M = M; g.N = N; g.K = K; g.batch = batch; g.opA = opA; g.opB = opB;
  g.A = (const cplx*)A; g.lda = lda; g.sA = sA;
  g.B = (const cplx*)B; g.ldb = ldb; g.sB = sB;
  g.C = (cplx*)C; g.ldc = ldc; g.sC = sC;
  g.alpha = cmk(1.0, 0.0); g.beta = cmk(0.0, 0.0);
  return zgemm_f64(g, (cudaStream_t)stream);
}

int ipeps_kernel_orth(int N, int k, int batch, const double* X, double* Q, int passes, int* fail_out,
                      void* stream) {
  if (N < k || k < 1 || batch < 1 || passes < 2 || !X || !Q) { set_thread_error("bad orth arguments"); return IPEPS_EINVAL; }
  if (!orth_supported(k)) { set_thread_error("orth: k too large"); return IPEPS_EUNSUPPORTED; }
  cudaStream_t st = (cudaStream_t)stream;
  const size_t wb = orth_work_bytes(N, k, batch);
  void* work = nullptr;
  int* dfail = nullptr;
  if (cudaMalloc(&work, wb) != cudaSuccess || cudaMalloc(&dfail, sizeof(int) * batch) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(work);
    set_thread_error("cudaMalloc failed");
    return IPEPS_ENOMEM;
  }
  int rc = 0;
  if (cudaMemsetAsync(dfail, 0, sizeof(int) * batch, st) != cudaSuccess)
    rc = cuda_fail(cudaGetLastError(), "orth fail flags", __FILE__, __LINE__);
  OrthDesc d;
  d.N = N; d.k = k; d.batch = batch;
  d.X = (const cplx*)X; d.sX = (long long)N * k; d.Q = (cplx*)Q; d.sQ = (long long)N * k;
  d.work = work; d.work_bytes = wb; d.skip = nullptr; d.fail = dfail; d.passes = passes; d.shifted = true;
  d.dev_fail = 1e-2;
  if (!rc) rc = orth_cqr(d, st);
  std::vector<int> hf(batch, 0);
  if (!rc && (cudaMemcpyAsync(hf.data(), dfail, sizeof(int) * batch, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
              cudaStreamSynchronize(st) != cudaSuccess))
    rc = cuda_fail(cudaGetLastError(), "orth sync", __FILE__, __LINE__);
  cudaFree(work);
  cudaFree(dfail);
  if (!rc && fail_out) memcpy(fail_out, hf.data(), sizeof(int) * batch);
  return rc;
}

int ipeps_kernel_gate(double J, double V, double h, double delta, double* out) {
  if (!out) { set_thread_error("out is NULL"); return IPEPS_EINVAL; }
  double* dbuf = nullptr;
  const int d = 4, d4 = d * d * d * d;
  if (cudaMalloc(&dbuf, sizeof(double) * (4 + 2 * d4)) != cudaSuccess) {
    cudaGetLastError();
    set_thread_error("cudaMalloc failed");
    return IPEPS_ENOMEM;
  }
  double hv[4] = {J, V, h, delta};
  int rc = 0;
  if (cudaMemcpy(dbuf, hv, sizeof(hv), cudaMemcpyHostToDevice) != cudaSuccess)
    rc = cuda_fail(cudaGetLastError(), "gate args", __FILE__, __LINE__);
  if (!rc) rc = build_gates(dbuf, dbuf + 1, dbuf + 2, dbuf + 3, 1, 1, d, 2, (cplx*)(dbuf + 4), 0);
  if (!rc && cudaMemcpy(out, dbuf + 4, sizeof(double) * 2 * d4, cudaMemcpyDeviceToHost) != cudaSuccess)
    rc = cuda_fail(cudaGetLastError(), "gate copy", __FILE__, __LINE__);
  cudaFree(dbuf);
  return rc;
}

static int split_hook(int op, int M, int N, int K, int batch, int opA, int opB, const double* A,
                      long long lda, long long sA, const double* B, long long ldb, long long sB,
                      double* C, long long ldc, long long sC, void* stream) {
  GemmDesc g;
  memset(&g, 0, sizeof(g));
  g.M = M; g.N = N; g.K = K; g.batch = batch; g.opA = opA; g.opB = opB;
  g.A = (const cplx*)A; g.lda = lda; g.sA = sA;
  g.B = (const cplx*)B; g.ldb = ldb; g.sB = sB;
  g.C = (cplx*)C; g.ldc = ldc; g.sC = sC;
  g.alpha = cmk(1.0, 0.0); g.beta = cmk(0.0, 0.0);
  const size_t bytes = tc::split_workspace_bytes(M, N, K, batch, op);
  void* work = nullptr;
  unsigned* derr = nullptr;
  if (cudaMalloc(&work, bytes) != cudaSuccess || cudaMalloc(&derr, sizeof(unsigned)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(work);
    set_thread_error("cudaMalloc failed");
    return IPEPS_ENOMEM;
  }
  cudaStream_t st = (cudaStream_t)stream;
  cudaMemsetAsync(derr, 0, sizeof(unsigned), st);
  int rc = tc::zgemm_split(g, op, work, bytes, derr, st);
  unsigned e = 0;
  if (!rc) {
    if (cudaMemcpyAsync(&e, derr, sizeof(unsigned), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      rc = cuda_fail(cudaGetLastError(), "split gemm sync", __FILE__, __LINE__);
  }
  cudaFree(work);
  cudaFree(derr);
  if (rc) return rc;
  if (e & DEV_TIMEOUT) { set_thread_error("tensor-core GEMM wait timed out"); return IPEPS_ETIMEOUT; }
  return 0;
}

int ipeps_kernel_zgemm_split(int M, int N, int K, int batch, int opA, int opB, const double* A,
                             long long lda, long long sA, const double* B, long long ldb, long long sB,
                             double* C, long long ldc, long long sC, void* stream) {
  return split_hook(tc::SPLIT_BF16, M, N, K, batch, opA, opB, A, lda, sA, B, ldb, sB, C, ldc, sC, stream);
}

int ipeps_kernel_zgemm_split_tf32(int M, int N, int K, int batch, int opA, int opB, const double* A,
                                  long long lda, long long sA, const double* B, long long ldb, long long sB,
                                  double* C, long long ldc, long long sC, void* stream) {
  return split_hook(tc::SPLIT_TF32, M, N, K, batch, opA, opB, A, lda, sA, B, ldb, sB, C, ldc, sC, stream);
}

int ipeps_kernel_permute(const double* in, double* out, int rank, const int* dims, const int* perm,
                         int batch, long long s_in, long long s_out, void* stream) {
  return permute_c128((const cplx*)in, (cplx*)out, rank, dims, perm, batch, s_in, s_out,
                      (cudaStream_t)stream);
}

int ipeps_kernel_svd(int m, int n, int batch, const double* A, double* U, double* S, double* V,
                     double tol, int max_sweeps, int* sweeps_out, void* stream) {
  if (m < n || n < 1 || batch < 1 || !A || !S) { set_thread_error("bad svd arguments"); return IPEPS_EINVAL; }
  if (!jacobi_svd_supported(m, n)) { set_thread_error("svd size too large"); return IPEPS_EUNSUPPORTED; }
  cudaStream_t st = (cudaStream_t)stream;
  // blocks too tall for shared memory keep their columns in a global-memory buffer
  cplx* gwork = nullptr;
  size_t gbytes = 0;
  if (!jacobi_svd_fits(m, n)) {
    gbytes = jacobi_svd_global_bytes(m, n, batch);
    if (cudaMalloc(&gwork, gbytes) != cudaSuccess) {
      cudaGetLastError();
      set_thread_error("cudaMalloc failed");
      return IPEPS_ENOMEM;
    }
  }
  std::vector<const void*> pa, pu, ps, pv;
  for (int b = 0; b < batch; ++b) {
    pa.push_back((const cplx*)A + (size_t)b * m * n);
    pu.push_back(U ? (void*)((cplx*)U + (size_t)b * m * n) : nullptr);
    ps.push_back(S + (size_t)b * n);
    pv.push_back(V ? (void*)((cplx*)V + (size_t)b * n * n) : nullptr);
  }
  void** dp = nullptr;
  unsigned* derr = nullptr;
  if (cudaMalloc(&dp, sizeof(void*) * 4 * batch) != cudaSuccess || cudaMalloc(&derr, sizeof(unsigned)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(gwork);
    set_thread_error("cudaMalloc failed");
    return IPEPS_ENOMEM;
  }
  std::vector<const void*> all;
  all.insert(all.end(), pa.begin(), pa.end());
  all.insert(all.end(), pu.begin(), pu.end());
  all.insert(all.end(), ps.begin(), ps.end());
  all.insert(all.end(), pv.begin(), pv.end());
  cudaMemcpy(dp, all.data(), sizeof(void*) * 4 * batch, cudaMemcpyHostToDevice);
  cudaMemset(derr, 0, sizeof(unsigned));
  SvdDesc d;
  d.m = m; d.n = n; d.batch = batch;
  d.A = (const cplx* const*)dp; d.lda = n;
  d.U = U ? (cplx* const*)(dp + batch) : nullptr; d.ldu = n;
  d.S = (double* const*)(dp + 2 * batch);
  d.V = V ? (cplx* const*)(dp + 3 * batch) : nullptr; d.ldv = n;
  d.tol = tol; d.max_sweeps = max_sweeps; d.err = derr; d.sweeps_out = sweeps_out; d.skip = nullptr;
  d.gwork = gwork; d.gwork_bytes = gbytes;
  int rc = jacobi_svd(d, st);
  unsigned e = 0;
  if (!rc) {
    cudaStreamSynchronize(st);
    cudaMemcpy(&e, derr, sizeof(unsigned), cudaMemcpyDeviceToHost);
  }
  cudaFree(dp);
  cudaFree(derr);
  cudaFree(gwork);
  if (rc) return rc;
  if (e & DEV_NONFINITE) { set_thread_error("non-finite input"); return IPEPS_ENAN; }
  if (e & DEV_JACOBI_CAP) { set_thread_error("sweep limit reached"); return IPEPS_ENOCONV; }
  return 0;
}

}  // extern "C"
