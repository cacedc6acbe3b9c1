// Library handle: all device state of `batch` independent iPEPS instances of equal shape.
#pragma once
#include <string>
#include <vector>

#include "arena.cuh"
#include "graph.cuh"
#include "linalg.cuh"
#include "su.cuh"

namespace ipeps {

constexpr int NPOS = 4;   // 2 x 2 unit cell, position index x + 2 y; A on x + y even

// Device pointer arrays of one directional left move (frame f, logical column x); each array is
// batched over (cut y, instance b) -> index y * B + b, or over corner slots (y * 4 + i) * B + b.
struct MovePlan {
  const cplx* const* g1A; const cplx* const* g1B; cplx* const* g1C;   // X1 = C T_cw      (8B)
  const cplx* const* g2A; const cplx* const* g2B; cplx* const* g2C;   // X2 = T_ccw X1    (8B)
  const cplx* const* g3B;                                             // rotated a_r      (8B)
  const cplx* const* hA; const cplx* const* hB; cplx* const* hC;      // halves           (4B)
  const cplx* const* c1A; const cplx* const* c1B;                     // C1' = P~[y-1] X1 (2B)
  const cplx* const* z1A; const cplx* const* z1B;                     // Z1 = T4 P[y-1]   (2B)
  const cplx* const* z2B;                                             // a(x, y)          (2B)
  const cplx* const* t4A;                                             // T4' = P~[y] Z2p  (2B)
  const cplx* const* w1A; const cplx* const* w1B;                     // W1 = T3 C4       (2B)
  const cplx* const* c4B;                                             // C4' = W1p P[y]   (2B)
  cplx* const* sC1; cplx* const* sT4; cplx* const* sC4;               // store targets    (2B)
};

// pool offsets of every pointer array, recorded while building and resolved after upload
struct MoveOff {
  size_t g1A, g1B, g1C, g2A, g2B, g2C, g3B, hA, hB, hC, c1A, c1B, z1A, z1B, z2B, t4A, w1A, w1B, c4B,
      sC1, sT4, sC4;
};
struct CtmOff {
  MoveOff mv[4][2];
  size_t csA, csS, pA, pU, pS, pV, envC, envT, yA, yU, yS, yV, zA, zU, zS, bA, bU;
};

struct CtmWork {
  cplx *X1, *X2, *X2p, *Y, *Q;       // corner pipeline [8B][...]
  cplx *H, *M;                       // halves [4B][N^2] (R~ then R), M [2B][N^2]
  cplx *U, *V; double* S;            // projector SVD [2B]
  cplx *Us, *Vs, *P, *Pt;            // [2B][N chi]
  cplx *Z1, *Z1p, *Z2, *Z2p, *T4n;   // edge absorption [2B]
  cplx *W1, *W1p, *C1n, *C4n;        // corner absorption [2B]
  int* kept;                         // [2B] projector rank
  // convergence
  double* cs;                        // [16B][chi] corner singular values of this sweep
  double* prev;                      // [16B][chi] normalised spectra of the previous sweep
  double* delta;                     // [B]
  int* frozen;                       // [B]
  int* sweeps;                       // [B]
  int* have_prev;                    // [1]
  double* best;                      // [B] best delta so far (stall test)
  int* since;                        // [B] sweeps without a factor-2 improvement of best
  const cplx* const* csA; double* const* csS;   // [16B] corner SVD operands
  // projector SVD operands [2B]
  const cplx* const* pA; cplx* const* pU; double* const* pS; cplx* const* pV;
  // environment slots in (kind, pos, b) order for the initial environment [4 NPOS B]
  cplx* const* envC; cplx* const* envT;
  // top-k projector SVD by subspace iteration (used when N > 2k): per (frame, column) slot the
  // converged right vectors are kept as the next call's starting block
  cplx* Vfin;                        // [4][2][2B][N k] right vectors per slot
  cplx *Vw, *Ysub, *Uy, *W, *Zsub, *Vz;   // [2B][N k] / [2B][k k]
  double *Sy, *Sz;                   // [2B][k]
  int* sub_done;                     // [2B] converged flags of the subspace iteration
  int* sub_rounds;                   // [2B] rounds used (diagnostics)
  double* sub_res;                   // [2B] previous residual (stagnation test)
  cplx* jgwork;                      // Jacobi column storage when N x k blocks exceed SMEM (or null)
  size_t jgwork_bytes;
  const cplx* const* yA; cplx* const* yU; double* const* yS; cplx* const* yV;   // Jacobi of Y
  const cplx* const* zA; cplx* const* zU; double* const* zS;                    // Jacobi of Z
  // Cholesky-QR subspace rounds (used when the k x k blocks fit; see subspace_svd)
  void* orth_work; size_t orth_bytes;
  cplx* Uq;                          // [2B][N k] orthonormal basis of Y
  cplx* Bk;                          // [2B][k k] Uq^+ Y
  cplx* Xk;                          // [2B][k k] left singular vectors of Bk
  cplx* part;                        // split-K partial products of Uq^+ Y
  int *ofail, *skip_new, *skip_old;  // [2B] per-problem path flags
  const cplx* const* bA; cplx* const* bU;                                        // Jacobi of Bk
};

struct Ctx {
  // parameters
  int B = 1, dA = 2, d = 4, D = 2, D2 = 4, chi = 8, N = 32, order = 1, precision = 0;
  int k = 32;              // projector subspace size (subspace_size)
  bool subspace = false;   // top-k subspace iteration instead of the full Jacobi SVD of M
  bool orth = false;       // subspace rounds by Cholesky QR + k x k Jacobi (else tall Jacobi)
  bool slot_warm[4][2] = {{false, false}, {false, false}, {false, false}, {false, false}};
  double dt = 0.02;
  double cut_rel = 1e-10;  // CTMRG projector truncation (relative)
  void* tcwork = nullptr;  // split-precision GEMM workspace (precision == 1)
  size_t tcwork_bytes = 0;
  unsigned long long seed = 0;
  std::vector<double> J, V, h;
  cudaStream_t st = nullptr;
  // memory
  Arena arena;
  PtrPool pool;
  void* dev_base = nullptr;
  void* dev_ptrs = nullptr;
  // state
  cplx *GA = nullptr, *GB = nullptr;
  double* lam = nullptr;
  double* eps = nullptr;
  double* dJ = nullptr; double* dV = nullptr; double* dh = nullptr; double* ddelta = nullptr;
  int ndelta = 0;
  std::vector<std::pair<int, int>> seq;   // Trotter sequence: (A's leg, delta index)
  cplx* gates = nullptr;                  // [B][ndelta][d^2][d^2]
  cplx* bondop = nullptr;                 // [B][d^2][d^2]
  SuWork su;
  cplx *Aph = nullptr, *Bph = nullptr;    // physical tensors [B][d][D^4]
  cplx* arot = nullptr;                   // double layers [site][rot][B][D2^4]
  cplx* Cenv[4][NPOS];                    // [B][chi][chi]
  cplx* Tenv[4][NPOS];                    // [B][chi][D2][chi]
  CtmWork w;
  MovePlan plan[4][2];
  CtmOff off;
  bool env_valid = false;
  double t = 0.0;
  unsigned* derr = nullptr;
  int* dflag = nullptr;                   // device scratch flag (all subspace problems converged)
  int* hflag = nullptr;                   // pinned host ints: [0] copy of dflag, [1] sweep limit
  // device-driven loops (graph.cuh): [0] sweep counter, [1] sweep limit, [2] subspace rounds
  int* loopctl = nullptr;
  GraphBuilder* gb = nullptr;             // non-null while a convergence graph is being captured
  bool graphs = true;                     // converge through one CUDA graph once the slots are warm
  cudaStream_t cap_st = nullptr;          // private stream the graph is captured on (st may be the
                                          // legacy default stream, which cannot capture)
  cudaGraphExec_t conv_exec = nullptr;    // cached convergence graph and the tolerance it was built for
  double conv_tol = 0.0;
  std::string msg;

  long long N2() const { return (long long)N * N; }
  long long D8() const { return (long long)D2 * D2 * D2 * D2; }
  cplx* a_rot(int site, int r) const { return arot + ((size_t)site * 4 + r) * B * D8(); }
};

// allocation / plan construction / execution (ctm.cu)
void ctm_carve(Ctx& c);
void ctm_build_plans(Ctx& c);            // record pointer arrays in the pool
void ctm_resolve_plans(Ctx& c);          // after the pool upload: device addresses
int ctm_prepare_tensors(Ctx& c);          // physical tensors + double layers from Gamma, lam
int ctm_init_env(Ctx& c);                 // traced double-layer start, zero-padded to chi
int ctm_sweep(Ctx& c);                    // one sweep: left, top, right, bottom moves
int ctm_spectra(Ctx& c, double tol, int first);   // corner spectra, delta, freeze converged

// Size of the projector subspace: chi + max(8, chi / 4) oversampling columns (at most N).  The
// top chi + 1 triplets converge at the rate (s_(k+1) / s_(chi+1))^2 per round, so the oversampling
// grows with chi, where spectra are flatter around the cut.
inline int subspace_size(int chi, int N) {
  const int over = chi / 4 > 8 ? chi / 4 : 8;
  return chi + over < N ? chi + over : N;
}

// Split-precision noise floors of the CTMRG convergence test: the smallest tolerance a split path
// honours (a smaller request is raised to it) and the stall threshold (a change that stops
// improving below it counts as stalled).  FP64: none and 1e-7.
inline double split_tol_floor(int precision) { return precision == 1 ? 1e-7 : precision == 2 ? 1e-8 : 0.0; }
inline double stall_threshold(int precision) { return precision == 1 ? 1e-5 : precision == 2 ? 1e-6 : 1e-7; }

// site type (0 = A, 1 = B) at a unit-cell position
__host__ __device__ inline int site_of(int pos) { return ((pos & 1) + (pos >> 1)) & 1; }
__host__ __device__ inline int pos_of(int x, int y) { return (x & 1) + 2 * (y & 1); }

}  // namespace ipeps
