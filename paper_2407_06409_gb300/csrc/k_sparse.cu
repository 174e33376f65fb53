// Block-sparse T_LR (Sec. III.A, Fig. sparsity).  The secondary cutoff leaves few site pairs of
// a sphere coupled when r_MBD,2 < r_MBD,1: the central row and column couple every site within
// r_MBD,1, any other pair only within r_MBD,2.  This path keeps, per central atom, the coupled
// pairs and their 3 x 3 blocks, and runs the Krylov chain and the adjoint pair products over
// them alone:
//   count    coupled partners of every site below and above it in the site order (before the
//            per-centre offsets, which then size the pair arrays)
//   prepare  blended polarisabilities (as in the dense path), the entries of every site's row,
//            the blocks and pair coefficients (FP64, blocks stored as float-float), v_1 = G e_k
//            and W_1 = D v_1
//   chain    v_{m+1} = D T W_m and W_{m+1} = D v_{m+1}: one thread per (site, column) over the
//            entries of the site's row in order (deterministic)
//   pair     M_st = P_s Q_t^T for the coupled pairs only, then the epilogue of the dense path
// FP64 runs at about 1/64 of the FP32 rate here, so the chain and pair products use
// float-float arithmetic (Dekker/Knuth error-free products and sums, about 2^-46 relative per
// product) on the FP32 pipe; the Krylov blocks leave it as FP64.
//
// Pattern test.  A pair is listed when its FP32 squared distance is below rc^2 (1 + 2e-4); the
// FP64 block of a listed pair is zero when its FP64 distance is not below rc, as in the dense
// path, so the slack adds explicit zero blocks only.  The sites of a centre are sorted by
// distance from it, so the partners of site s within r lie among the sites whose radius differs
// from r_s by less than r: a window found by binary search, with a further 2e-3 bohr of slack.
#include "ff.cuh"
#include "lmbd_internal.cuh"
#include "pair_epilogue.cuh"

#define SP_THREADS 256
#define SP_WARPS (SP_THREADS / 32)

struct SpCut {
  float c1, c2;   // squared cutoffs with slack (bohr^2): central pairs, other pairs
  float w1, w2;   // radius windows (bohr): r_MBD,1 and r_MBD,2 with slack
};

__device__ __forceinline__ SpCut sp_cut(const DevParams& p) {
  SpCut k;
  k.c1 = __double2float_rn(p.r_mbd1 * p.r_mbd1 * (1.0 + 2e-4));
  k.c2 = __double2float_rn(p.r_mbd2 * p.r_mbd2 * (1.0 + 2e-4));
  k.w1 = __double2float_rn(p.r_mbd1 * (1.0 + 1e-4) + 2e-3);
  k.w2 = __double2float_rn(p.r_mbd2 * (1.0 + 1e-4) + 2e-3);
  return k;
}

// xf[s] = (x, y, z, |x|) of every site in FP32.
__device__ __forceinline__ void sp_load_sites(const Work& w, int c, int ns, float4* xf) {
  const long long sbase = (long long)c * w.site_cap;
  for (int s = threadIdx.x; s < ns; s += blockDim.x) {
    const double x0 = w.site_x[3 * (sbase + s)], x1 = w.site_x[3 * (sbase + s) + 1], x2 = w.site_x[3 * (sbase + s) + 2];
    xf[s] = make_float4(__double2float_rn(x0), __double2float_rn(x1), __double2float_rn(x2),
                        __double2float_rn(sqrt(x0 * x0 + x1 * x1 + x2 * x2)));
  }
}

// The pattern test, symmetric in (s, t) bit for bit (differences change sign only, and the
// products and sums are rounded one by one).
__device__ __forceinline__ bool sp_couple(const float4* xf, int s, int t, const SpCut& k) {
  const float dx = __fsub_rn(xf[t].x, xf[s].x), dy = __fsub_rn(xf[t].y, xf[s].y), dz = __fsub_rn(xf[t].z, xf[s].z);
  const float d2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
  return d2 < ((s == 0 || t == 0) ? k.c1 : k.c2);
}

// first i in [lo, hi) with radius >= v, and first i in [lo, hi) with radius > v
__device__ __forceinline__ int sp_lower(const float4* xf, int lo, int hi, float v) {
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (xf[mid].w < v) lo = mid + 1; else hi = mid;
  }
  return lo;
}
__device__ __forceinline__ int sp_upper(const float4* xf, int lo, int hi, float v) {
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (xf[mid].w <= v) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// The coupled partners of site s below it (upper = false; the central site first) or above it
// (upper = true), ascending, one warp: f(t, rank) once per partner, rank counted from 0 within
// the part.  Returns the number of partners in the part.
template <class F>
__device__ __forceinline__ int sp_scan(const float4* xf, int ns, int s, bool upper, const SpCut& k, F&& f) {
  const int lane = threadIdx.x & 31;
  int b, e, n = 0;
  if (!upper) {
    if (s == 0) return 0;
    if (sp_couple(xf, s, 0, k)) {
      if (lane == 0) f(0, 0);
      n = 1;
    }
    b = sp_lower(xf, 1, s, xf[s].w - k.w2);
    e = s;
  } else {
    b = s + 1;
    e = s == 0 ? sp_upper(xf, 1, ns, k.w1) : sp_upper(xf, s + 1, ns, xf[s].w + k.w2);
  }
  for (int t0 = b; t0 < e; t0 += 32) {
    const int t = t0 + lane;
    const bool hit = t < e && sp_couple(xf, s, t, k);
    const unsigned m = __ballot_sync(0xffffffffu, hit);
    if (hit) f(t, n + __popc(m & ((1u << lane) - 1u)));
    n += __popc(m);
  }
  return n;
}

// ---------------------------------------------------------------------------------------
// count: sp_cnt[c][s] = (partners below s, partners above s), sp_np[c] = coupled pairs
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(SP_THREADS) k_sp_count(Work w, DevParams p) {
  extern __shared__ float4 sp_xf[];
  __shared__ int tot[SP_WARPS];
  const int c = blockIdx.x;
  const int ns = min(w.counts[c].ns, w.site_cap);
  const SpCut k = sp_cut(p);
  sp_load_sites(w, c, ns, sp_xf);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int mine = 0;
  for (int s = warp; s < ns; s += SP_WARPS) {
    const int L = sp_scan(sp_xf, ns, s, false, k, [](int, int) {});
    const int U = sp_scan(sp_xf, ns, s, true, k, [](int, int) {});
    if (lane == 0) w.sp_cnt[(long long)c * w.site_cap + s] = make_int2(L, U);
    mine += L;
  }
  if (lane == 0) tot[warp] = mine;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int i = 0; i < SP_WARPS; ++i) t += tot[i];
    w.sp_np[c] = t;
  }
}

// Exclusive prefix sums of a[0..n) and b[0..n) in place (one block); a[n], b[n] = the totals.
__device__ void sp_block_scan2(int* a, int* b, int n) {
  __shared__ int wa[SP_WARPS], wb[SP_WARPS];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int per = (n + blockDim.x - 1) / blockDim.x;
  const int i0 = min(n, tid * per), i1 = min(n, i0 + per);
  int sa = 0, sb = 0;
  for (int i = i0; i < i1; ++i) {
    sa += a[i];
    sb += b[i];
  }
  int xa = sa, xb = sb;   // inclusive warp scan
  for (int o = 1; o < 32; o <<= 1) {
    const int ya = __shfl_up_sync(0xffffffffu, xa, o), yb = __shfl_up_sync(0xffffffffu, xb, o);
    if (lane >= o) {
      xa += ya;
      xb += yb;
    }
  }
  if (lane == 31) {
    wa[warp] = xa;
    wb[warp] = xb;
  }
  __syncthreads();
  int ba = 0, bb = 0;
  for (int v = 0; v < warp; ++v) {
    ba += wa[v];
    bb += wb[v];
  }
  int ra = ba + xa - sa, rb = bb + xb - sb;   // exclusive start of this thread's chunk
  for (int i = i0; i < i1; ++i) {
    const int va = a[i], vb = b[i];
    a[i] = ra;
    b[i] = rb;
    ra += va;
    rb += vb;
  }
  if (tid == blockDim.x - 1) {
    a[n] = ra;
    b[n] = rb;
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------------------
// prepare: one block per central atom
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(SP_THREADS) k_sp_prepare(Work w, DevParams p, int c0, int max_ns) {
  extern __shared__ double sp_smem[];
  const int c = c0 + blockIdx.x;
  if (c >= w.n_atoms) return;
  const Counts cn = w.counts[c];
  const int ns = cn.ns, n1 = cn.n1;
  const int ms = (max_ns + 1) & ~1;
  double* rt = sp_smem;                                     // ms
  float4* xf = reinterpret_cast<float4*>(rt + ms);          // ms
  int* rs = reinterpret_cast<int*>(xf + ms);                // ms + 1: first entry of each row
  int* pb = rs + ms + 1;                                    // ms + 1: first pair of each row
  int* lc = pb + ms + 1;                                    // ms: partners below each site
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long long sbase = (long long)c * w.site_cap;
  const long long offs = w.off_s[c], offk1 = w.off_k1[c];
  const long long pbg = w.off_np[c], eb = 2 * pbg;
  const int np = (int)(w.off_np[c + 1] - pbg);
  const SpCut k = sp_cut(p);
  sp_load_sites(w, c, ns, xf);
  for (int s = tid; s < ns; s += blockDim.x) {
    const int a = w.site_atom[sbase + s];
    const double x0 = w.site_x[3 * (sbase + s)], x1 = w.site_x[3 * (sbase + s) + 1], x2 = w.site_x[3 * (sbase + s) + 2];
    rt[s] = mbd_blend_site(w, p, s, a, n1, offs, offk1, x0, x1, x2);
    for (int q = 0; q < p.nq; ++q) {
      const ff d = ff_from_double(w.dsq[(offs + s) * p.nq + q]);
      w.dsq_ff[(offs + s) * p.nq + q] = make_float2(d.hi, d.lo);
    }
    const int2 cnt = w.sp_cnt[sbase + s];
    rs[s] = cnt.x + cnt.y;
    pb[s] = cnt.x;
    lc[s] = cnt.x;
  }
  __syncthreads();
  sp_block_scan2(rs, pb, ns);
  if (pb[ns] != np || rs[ns] != 2 * np) {   // counts of another site list: nothing is written
    if (tid == 0) atomicOr(w.status, LMBD_FLAG_PATTERN);
    return;
  }
  for (int s = tid; s < ns; s += blockDim.x) w.sp_row[offs + s] = make_int4(rs[s], rs[s + 1] - rs[s], pb[s], lc[s]);
  // partners below each site: entries (t, pair) and the pair list, pairs in row order
  for (int s = warp; s < ns; s += SP_WARPS) {
    const int L = lc[s], start = rs[s], base = pb[s];
    const int n = sp_scan(xf, ns, s, false, k, [&](int t, int r) {
      if (r < L) {
        w.sp_ent[eb + start + r] = make_int2(t, base + r);
        w.sp_pair[pbg + base + r] = make_int2(s, t);
      }
    });
    if (n != L && lane == 0) atomicOr(w.status, LMBD_FLAG_PATTERN);
  }
  __syncthreads();
  // blocks and pair coefficients, one thread per pair
  for (int i = tid; i < np; i += blockDim.x) {
    const int2 st = w.sp_pair[pbg + i];
    const double* xs = w.site_x + 3 * (sbase + st.x);
    const double* xt = w.site_x + 3 * (sbase + st.y);
    const double rr[3] = {xt[0] - xs[0], xt[1] - xs[1], xt[2] - xs[2]};
    double blk[3][3], kc[5];
    tlr_pair_block(p, rr, st.y == 0 ? p.r_mbd1 : p.r_mbd2, rt[st.x], rt[st.y], blk, w.pcoef ? kc : nullptr);
    const ff b00 = ff_from_double(blk[0][0]), b11 = ff_from_double(blk[1][1]), b22 = ff_from_double(blk[2][2]);
    const ff b01 = ff_from_double(blk[0][1]), b02 = ff_from_double(blk[0][2]), b12 = ff_from_double(blk[1][2]);
    float4* b = w.sp_blk + 3 * (pbg + i);
    b[0] = make_float4(b00.hi, b00.lo, b11.hi, b11.lo);
    b[1] = make_float4(b22.hi, b22.lo, b01.hi, b01.lo);
    b[2] = make_float4(b02.hi, b02.lo, b12.hi, b12.lo);
    if (w.pcoef) {
      double* pc = w.pcoef + 8 * (pbg + i);
      pc[0] = rr[0]; pc[1] = rr[1]; pc[2] = rr[2];
      pc[3] = kc[0]; pc[4] = kc[1]; pc[5] = kc[2]; pc[6] = kc[3]; pc[7] = kc[4];
    }
  }
  // partners above each site: the pair (t, s), t > s, is the entry of s among the partners
  // below t (ascending there, found by binary search)
  for (int s = warp; s < ns; s += SP_WARPS) {
    const int L = lc[s], U = rs[s + 1] - rs[s] - L, start = rs[s] + L;
    const int n = sp_scan(xf, ns, s, true, k, [&](int t, int r) {
      if (r >= U) return;
      const int2* row = w.sp_ent + eb + rs[t];
      int lo = 0, hi = lc[t];
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (row[mid].x < s) lo = mid + 1; else hi = mid;
      }
      int pid = 0;
      if (lo < lc[t] && row[lo].x == s) pid = row[lo].y;
      else atomicOr(w.status, LMBD_FLAG_PATTERN);
      w.sp_ent[eb + start + r] = make_int2(t, pid);
    });
    if (n != U && lane == 0) atomicOr(w.status, LMBD_FLAG_PATTERN);
  }
  __syncthreads();
  // v_1 = G e_k = D T_{s0} D_0 (the central partner is the first entry of a row) and W_1 = D v_1
  const int ncv = 3 * p.n_freq;
  double* V1 = w.vkr + (offs * 3) * ncv;
  float2* W1 = w.wff + (offs * 3) * ncv;
  for (int e = tid; e < 3 * ns * ncv; e += blockDim.x) {
    const int row = e / ncv, col = e % ncv;
    const int s = row / 3, al = row % 3, q = col / 3 + 1, be = col % 3;
    const double ds = w.dsq[(offs + s) * p.nq + q];
    double v = 0.0;
    if (s > 0 && lc[s] > 0 && w.sp_ent[eb + rs[s]].x == 0) {
      const int slot = al == be ? al : al + be + 2;   // (01) 3, (02) 4, (12) 5
      const float2 tb = reinterpret_cast<const float2*>(w.sp_blk + 3 * (pbg + pb[s]))[slot];
      v = ds * w.dsq[offs * p.nq + q] * ((double)tb.x + (double)tb.y);
    }
    V1[(long long)row * ncv + col] = v;
    const ff wv = ff_from_double(ds * v);
    W1[(long long)row * ncv + col] = make_float2(wv.hi, wv.lo);
  }
}

// acc += a b in float-float (a = (ah, al)): exact product of the leading parts by an FMA, the
// cross terms in FP32, the leading sum by an error-free two-sum; the low part is renormalised
// when the result leaves float-float.
__device__ __forceinline__ void ffmac(ff& acc, float ah, float al, float2 b) {
  const float pr = __fmul_rn(ah, b.x);
  float e = __fmaf_rn(ah, b.x, -pr);
  e = __fmaf_rn(ah, b.y, e);
  e = __fmaf_rn(al, b.x, e);
  const float s = __fadd_rn(acc.hi, pr);
  const float bb = __fsub_rn(s, acc.hi);
  const float err = __fadd_rn(__fsub_rn(acc.hi, __fsub_rn(s, bb)), __fsub_rn(pr, bb));
  acc.hi = s;
  acc.lo = __fadd_rn(acc.lo, __fadd_rn(err, e));
}

// ---------------------------------------------------------------------------------------
// chain step m: v_{m+1} = D (T W_m), W_{m+1} = D v_{m+1}; rpb sites per block, one thread per
// (site, column); W_m is block m - 1 of wff (all blocks kept for the adjoint)
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(SP_THREADS) k_sp_chain(Work w, DevParams p, int m, int c0, int bpc, int rpb) {
  const int c = c0 + blockIdx.x / bpc;
  if (c >= w.n_atoms) return;
  const int ns = w.counts[c].ns;
  const int s0 = (blockIdx.x % bpc) * rpb;
  if (s0 >= ns) return;
  const int ncv = 3 * p.n_freq;
  const long long offs = w.off_s[c], pbg = w.off_np[c], eb = 2 * pbg;
  const float2* Win = w.wff + (long long)(m - 1) * w.vstride;
  float2* Wout = w.wff + (long long)m * w.vstride;
  double* Vout = w.vkr + (long long)m * w.vstride + (offs * 3) * ncv;
  for (int it = threadIdx.x; it < rpb * ncv; it += blockDim.x) {
    const int s = s0 + it / ncv, col = it % ncv;
    if (s >= ns) break;
    const int4 row = w.sp_row[offs + s];
    const int2* ent = w.sp_ent + eb + row.x;
    ff a0 = ff_make(0.f, 0.f), a1 = a0, a2 = a0;
    for (int e = 0; e < row.y; ++e) {
      const int2 en = ent[e];
      const float4* b = w.sp_blk + 3 * (pbg + en.y);
      const float4 b0 = b[0], b1 = b[1], b2 = b[2];   // (00, 11), (22, 01), (02, 12)
      const float2* x = Win + ((offs + en.x) * 3) * ncv + col;
      const float2 x0 = x[0], x1 = x[ncv], x2 = x[2 * ncv];
      ffmac(a0, b0.x, b0.y, x0);
      ffmac(a0, b1.z, b1.w, x1);
      ffmac(a0, b2.x, b2.y, x2);
      ffmac(a1, b1.z, b1.w, x0);
      ffmac(a1, b0.z, b0.w, x1);
      ffmac(a1, b2.z, b2.w, x2);
      ffmac(a2, b2.x, b2.y, x0);
      ffmac(a2, b2.z, b2.w, x1);
      ffmac(a2, b1.x, b1.y, x2);
    }
    // v = D y and W = D v in float-float; one FP64 sum per output for the FP64 Krylov block
    const float2 dq = w.dsq_ff[(offs + s) * p.nq + col / 3 + 1];
    const ff d = ff_make(dq.x, dq.y);
    const ff acc[3] = {a0, a1, a2};
#pragma unroll
    for (int al = 0; al < 3; ++al) {
      const ff v = ff_mul(d, ff_quick_two_sum(acc[al].hi, acc[al].lo));
      Vout[(long long)(3 * s + al) * ncv + col] = (double)v.hi + (double)v.lo;
      const ff wv = ff_mul(d, v);
      Wout[((offs + s) * 3 + al) * ncv + col] = make_float2(wv.hi, wv.lo);
    }
  }
}

// ---------------------------------------------------------------------------------------
// adjoint pair products: 256 pairs per block, 32 per warp.  Eight lanes share a pair's inner
// product over the ncol columns (four pairs at a time), then each lane takes one pair of the
// warp through the FP64 epilogue and the gradient atomics.
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(SP_THREADS) k_sp_adj_pair(Work w, DevParams p, int c0, int bpc) {
  __shared__ float2 accs[SP_WARPS][32][9];
  const int c = c0 + blockIdx.x / bpc;
  if (c >= w.n_atoms) return;
  const long long pbg = w.off_np[c];
  const int np = (int)(w.off_np[c + 1] - pbg);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int j0 = (blockIdx.x % bpc) * SP_THREADS + warp * 32;
  if (j0 >= np) return;
  const long long offs = w.off_s[c];
  const int ncol = w.ncol;
  const int g = lane >> 3, l = lane & 7;
  for (int r = 0; r < 8; ++r) {
    const int j = j0 + 4 * r + g;
    ff acc[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) acc[i] = ff_make(0.f, 0.f);
    if (j < np) {
      const int2 st = w.sp_pair[pbg + j];
      const float2* P = w.pff + (offs * 3 + 3 * st.x) * (long long)ncol;
      const float2* Q = w.qff + (offs * 3 + 3 * st.y) * (long long)ncol;
      for (int k = l; k < ncol; k += 8) {
        const float2 p0 = P[k], p1 = P[ncol + k], p2 = P[2 * ncol + k];
        const float2 q0 = Q[k], q1 = Q[ncol + k], q2 = Q[2 * ncol + k];
        ffmac(acc[0], p0.x, p0.y, q0);
        ffmac(acc[1], p0.x, p0.y, q1);
        ffmac(acc[2], p0.x, p0.y, q2);
        ffmac(acc[3], p1.x, p1.y, q0);
        ffmac(acc[4], p1.x, p1.y, q1);
        ffmac(acc[5], p1.x, p1.y, q2);
        ffmac(acc[6], p2.x, p2.y, q0);
        ffmac(acc[7], p2.x, p2.y, q1);
        ffmac(acc[8], p2.x, p2.y, q2);
      }
    }
#pragma unroll
    for (int o = 1; o < 8; o <<= 1)
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        const ff other = ff_make(__shfl_xor_sync(0xffffffffu, acc[i].hi, o), __shfl_xor_sync(0xffffffffu, acc[i].lo, o));
        acc[i] = ff_add(acc[i], other);
      }
#pragma unroll
    for (int i = 0; i < 9; ++i)
      if (i == l || (l == 0 && i == 8)) accs[warp][4 * r + g][i] = make_float2(acc[i].hi, acc[i].lo);
  }
  __syncwarp();
  const int j = j0 + lane;
  if (j >= np) return;
  const int2 st = w.sp_pair[pbg + j];
  double a[3][3];
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const float2 v = accs[warp][lane][i];
    a[i / 3][i % 3] = (double)v.x + (double)v.y;
  }
  double out[4];
  pair_epilogue_at(w, offs, w.pcoef + 8 * (pbg + j), st.x, st.y, a, out);
  const long long sbase = (long long)c * w.site_cap;
  if (out[0] != 0.0 || out[1] != 0.0 || out[2] != 0.0) {
    const int as = w.site_atom[sbase + st.x], at = w.site_atom[sbase + st.y];
    atomic_add3(w.gacc + 3 * at, out[0], out[1], out[2]);
    atomic_add3(w.gacc + 3 * as, -out[0], -out[1], -out[2]);
  }
  if (out[3] != 0.0) {
    atomicAdd(&w.rbar[offs + st.x], out[3]);
    atomicAdd(&w.rbar[offs + st.y], out[3]);
  }
}

// ---------------------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------------------
void launch_sp_count(const Work& w, const DevParams& p, cudaStream_t s) {
  if (w.n_atoms == 0) return;
  const size_t sm = sizeof(float4) * (size_t)w.site_cap;
  raise_smem_limit((const void*)k_sp_count, sm);
  k_sp_count<<<w.n_atoms, SP_THREADS, sm, s>>>(w, p);
}

void launch_sp_prepare(const Work& w, const DevParams& p, int c0, int c1, int max_ns, cudaStream_t s) {
  if (c1 <= c0) return;
  const size_t ms = (size_t)((max_ns + 1) & ~1);
  const size_t sm = sizeof(double) * ms + sizeof(float4) * ms + sizeof(int) * (3 * ms + 2);
  raise_smem_limit((const void*)k_sp_prepare, sm);
  k_sp_prepare<<<c1 - c0, SP_THREADS, sm, s>>>(w, p, c0, max_ns);
}

void launch_sp_chain(const Work& w, const DevParams& p, int m, int c0, int c1, int max_ns, cudaStream_t s) {
  if (c1 <= c0 || max_ns <= 0) return;
  const int ncv = 3 * p.n_freq;
  const int rpb = ncv >= SP_THREADS ? 1 : SP_THREADS / ncv;
  const int bpc = (max_ns + rpb - 1) / rpb;
  k_sp_chain<<<(c1 - c0) * bpc, SP_THREADS, 0, s>>>(w, p, m, c0, bpc, rpb);
}

void launch_sp_adj_pair(const Work& w, const DevParams& p, int c0, int c1, int max_pairs, cudaStream_t s) {
  if (c1 <= c0 || max_pairs <= 0) return;
  const int bpc = (max_pairs + SP_THREADS - 1) / SP_THREADS;
  k_sp_adj_pair<<<(c1 - c0) * bpc, SP_THREADS, 0, s>>>(w, p, c0, bpc);
}
