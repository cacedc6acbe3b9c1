// Readout work buffers and driver (see measure.cu).
#pragma once
#include "arena.cuh"
#include "linalg.cuh"

namespace ipeps {
struct Ctx;

// The eight left halves per instance are 8 B independent jobs (frame, site, instance); their
// large intermediates (tl, W1, bl, W2, W2p, X, Y) are held for `group` jobs at a time and the jobs
// run in passes of that many, so the readout workspace stays bounded (kMeasurePassBytes) however
// large D, chi and B are.  The single layers ak, akc, the left halves Lh and everything after them
// hold all 8 B jobs.
struct MeasureWork {
  cplx *tl, *W1, *bl, *W2, *W2p, *X, *Y, *ak, *akc, *Lh, *RCt, *RC, *rho1, *rho2;
  double* obs;
  int group;                // jobs per pass
};
constexpr size_t kMeasurePassBytes = size_t(4) << 30;
int measure_group(int B, int d, int D, int chi);
struct MeasureOff { size_t tlA, tlB, w1A, blA, blB, aoB, rcA, rcB, rcC, r1, r2; };
struct MeasurePlan {
  const cplx* const* tlA; const cplx* const* tlB; const cplx* const* w1A;
  const cplx* const* blA; const cplx* const* blB; const cplx* const* aoB;
  const cplx* const* rcA; const cplx* const* rcB; const cplx* const* rcC;
  const cplx* const* r1; const cplx* const* r2;
};

size_t measure_bytes(int B, int d, int D, int chi);
void measure_carve(Arena& a, MeasureWork& w, int B, int d, int D, int chi);
void measure_build(Ctx& c, MeasureWork& w, PtrPool& pool, MeasureOff& o);
void measure_resolve(const PtrPool& P, const MeasureOff& o, MeasurePlan& m);
constexpr int kObsPerInstance = 11;
// fills host_out[b * kObsPerInstance + {nA, nB, I, tauzA, tauzB, energy, purityA, tr_rhoA,
// S1_A, S1/2_A, S2_A}] (Renyi entropies of the physical one-site RDM of A)
int measure_run(Ctx& c, MeasureWork& w, const MeasurePlan& m, double* host_out);
}  // namespace ipeps
