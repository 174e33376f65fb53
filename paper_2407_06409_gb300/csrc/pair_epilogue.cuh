// Per-pair epilogue of the adjoint pair-matrix contraction (shared by the FP64, warp-level
// and tcgen05 pair kernels).
#pragma once
#include "lmbd_internal.cuh"

// Contribution of the site pair (s, t), s > t, to dL/dr and dL/dR~ from its pair-matrix
// block acc = M_st (3 x 3, before the central-column term): T_LR,st = f_LR f(r, S~) T(r), with
// pc the pair's geometry and derivative coefficients (r (3), k1..k5, written by the prepare
// kernels).  Returns g = dL/dr_t (= -dL/dr_s) in out[0..2] and the SCS-radius seed
// beta dL/dS~ in out[3] (zeros when the pair does not couple).
__device__ __forceinline__ void pair_epilogue_at(const Work& w, long long offs, const double* pc, int s, int t,
                                                 double (&acc)[3][3], double* out) {
  out[0] = out[1] = out[2] = out[3] = 0.0;
  const double k3 = pc[5];
  if (k3 == 0.0 && pc[6] == 0.0) return;
  if (t == 0) {
    const double* x0 = w.x0buf + (offs + s) * 9;
#pragma unroll
    for (int al = 0; al < 3; ++al)
#pragma unroll
      for (int be = 0; be < 3; ++be) acc[al][be] += x0[al * 3 + be];
  }
  const double rr[3] = {pc[0], pc[1], pc[2]};
  const double M[6] = {acc[0][0], acc[1][1], acc[2][2], 0.5 * (acc[0][1] + acc[1][0]),
                       0.5 * (acc[0][2] + acc[2][0]), 0.5 * (acc[1][2] + acc[2][1])};
  const double Mr[3] = {M[0] * rr[0] + M[3] * rr[1] + M[4] * rr[2], M[3] * rr[0] + M[1] * rr[1] + M[5] * rr[2],
                        M[4] * rr[0] + M[5] * rr[1] + M[2] * rr[2]};
  const double trM = M[0] + M[1] + M[2];
  const double rMr = rr[0] * Mr[0] + rr[1] * Mr[1] + rr[2] * Mr[2];
  const double radial = pc[3] * rMr + pc[4] * trM;
  out[0] = radial * rr[0] + k3 * Mr[0];
  out[1] = radial * rr[1] + k3 * Mr[1];
  out[2] = radial * rr[2] + k3 * Mr[2];
  out[3] = pc[6] * rMr + pc[7] * trM;
}

// The pair (s, t) of the dense pair-coefficient layout (lower triangle, s (s - 1) / 2 + t).
__device__ __forceinline__ void pair_epilogue(const Work& w, long long offs, long long offt, int s, int t, int ns,
                                              double (&acc)[3][3], double* out) {
  if (!(s < ns && t < ns && s > t)) {
    out[0] = out[1] = out[2] = out[3] = 0.0;
    return;
  }
  pair_epilogue_at(w, offs, w.pcoef + offt + 8LL * (s * (s - 1) / 2 + t), s, t, acc, out);
}
