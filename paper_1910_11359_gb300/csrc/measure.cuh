// Readout work buffers and driver (see measure.cu).
#pragma once
#include "arena.cuh"
#include "linalg.cuh"

namespace ipeps {
struct Ctx;

struct MeasureWork {
  cplx *tl, *W1, *bl, *W2, *W2p, *ao, *Lh, *RCt, *RC, *rho1, *rho2;
  double* obs;
};
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
