// Neighbour search: free-atom quantities, cell list, per-centre site lists.
//
// A site is an atom together with a lattice shift (Sec. III.A: replicas are
// captured in real space, so every periodic image inside a radius is its own
// site).  Each central atom k gets the sites within
// r_list = max(2 r_SCS, sphere radius), sorted by distance, so that
//   K1 (r < r_SCS), the MBD sphere (r < r_sphere) and K1 u K2 (r < 2 r_SCS)
// are prefixes of one list (Sec. III.A and III.B).  Set membership compares
// squared distances in Angstrom against squared radii in Angstrom.
#include "lmbd_internal.cuh"

// ---------------------------------------------------------------------------------------
// free-atom quantities (Sec. II.B): alpha_bar_i(omega) = alpha0 nu / (1 + (omega/omega_i)^2),
// omega_i = 4 C6 / (3 alpha0^2), sigma_i = (sqrt(2/pi) alpha_bar / 3)^(1/3), R_i = R0 nu^(1/3)
// ---------------------------------------------------------------------------------------
__global__ void k_free_atom(Work w, DevParams p) {
  int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= w.n_atoms) return;
  int s = w.species[a];
  double nu = w.nu[a];
  // device-resident inputs are validated here (host arrays are checked before the copy): a
  // species index outside the table is never used to index it; the call then returns
  // LMBD_EINVAL after the neighbour phase
  const bool bad = s < 0 || s >= p.n_species || !(nu > 0.0) || !isfinite(nu) || !isfinite(w.pos[3 * a]) ||
                   !isfinite(w.pos[3 * a + 1]) || !isfinite(w.pos[3 * a + 2]);
  if (bad) {
    atomicOr(w.status, LMBD_FLAG_BAD_INPUT);
    s = 0;
    nu = 1.0;
  }
  double a0 = w.table[3 * s + 0], c6 = w.table[3 * s + 1], r0 = w.table[3 * s + 2];
  double om = 4.0 * c6 / (3.0 * a0 * a0);
  const double c = 0.26596152026762182;  // sqrt(2/pi)/3
  for (int q = 0; q < p.nqs; ++q) {   // at the frequencies of the SCS solves
    double u = p.omega_s[q] / om;
    double ab = a0 * nu / (1.0 + u * u);
    w.abar[a * p.nqs + q] = ab;
    w.sig[a * p.nqs + q] = cbrt(c * ab);
  }
  w.rvdw[a] = r0 * cbrt(nu);
  w.a0[a] = a0;
  w.r0[a] = r0;
}

void launch_free_atom(const Work& w, const DevParams& p, cudaStream_t s) {
  if (w.n_atoms == 0) return;
  k_free_atom<<<(w.n_atoms + 127) / 128, 128, 0, s>>>(w, p);
}

// ---------------------------------------------------------------------------------------
// cell list
// ---------------------------------------------------------------------------------------
// Non-periodic structures: bounding box and grid, computed on the device by one block.
__global__ void k_bbox(Work w, Grid* g, double r_list) {
  __shared__ double lo[3][256], hi[3][256];
  double l[3] = {1e300, 1e300, 1e300}, h[3] = {-1e300, -1e300, -1e300};
  for (int a = threadIdx.x; a < w.n_atoms; a += blockDim.x)
    for (int d = 0; d < 3; ++d) {
      double v = w.pos[3 * a + d];
      l[d] = fmin(l[d], v);
      h[d] = fmax(h[d], v);
    }
  for (int d = 0; d < 3; ++d) { lo[d][threadIdx.x] = l[d]; hi[d][threadIdx.x] = h[d]; }
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st)
      for (int d = 0; d < 3; ++d) {
        lo[d][threadIdx.x] = fmin(lo[d][threadIdx.x], lo[d][threadIdx.x + st]);
        hi[d][threadIdx.x] = fmax(hi[d][threadIdx.x], hi[d][threadIdx.x + st]);
      }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    for (int d = 0; d < 3; ++d) {
      double ext = hi[d][0] - lo[d][0];
      int nc = (int)(ext / r_list);
      if (nc < 1) nc = 1;
      if (nc > 64) nc = 64;
      double hh = ext / nc;
      if (hh < r_list) hh = r_list;     // every cell at least r_list wide
      g->origin[d] = lo[d][0];
      g->h[d] = hh;
      g->nc[d] = nc;
      g->reach[d] = 1;
    }
  }
}

// Fractional coordinates f in [0, 1) of atom a, its wrapped position wpos = f C and the lattice
// translation wrap = floor(frac) with pos = wpos + wrap C (periodic structures).
__device__ __forceinline__ void wrap_position(const Work& w, const Grid& g, int a, const double* x, double* f) {
  for (int d = 0; d < 3; ++d) {
    double v = x[0] * g.inv[0 * 3 + d] + x[1] * g.inv[1 * 3 + d] + x[2] * g.inv[2 * 3 + d];
    double fl = floor(v);
    v -= fl;
    if (v >= 1.0) {
      v = 0.0;
      fl += 1.0;
    }
    f[d] = v;
    w.wrap[3 * a + d] = (int)fl;
  }
  for (int d = 0; d < 3; ++d)
    w.wpos[3 * a + d] = f[0] * g.cell[0 * 3 + d] + f[1] * g.cell[1 * 3 + d] + f[2] * g.cell[2 * 3 + d];
}

// Wrapped positions only (site lists refreshed from a resident candidate list).
__global__ void k_wrap(Work w, const Grid* __restrict__ gp) {
  int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= w.n_atoms) return;
  const Grid& g = *gp;
  double x[3] = {w.pos[3 * a], w.pos[3 * a + 1], w.pos[3 * a + 2]};
  if (g.periodic) {
    double f[3];
    wrap_position(w, g, a, x, f);
  } else {
    for (int d = 0; d < 3; ++d) {
      w.wpos[3 * a + d] = x[d];
      w.wrap[3 * a + d] = 0;
    }
  }
}

__global__ void k_bin(Work w, const Grid* __restrict__ gp) {
  int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= w.n_atoms) return;
  const Grid& g = *gp;
  double x[3] = {w.pos[3 * a], w.pos[3 * a + 1], w.pos[3 * a + 2]};
  int ci[3];
  if (g.periodic) {
    double f[3];
    wrap_position(w, g, a, x, f);
    for (int d = 0; d < 3; ++d) {
      int c = (int)(f[d] * g.nc[d]);
      ci[d] = c < 0 ? 0 : (c >= g.nc[d] ? g.nc[d] - 1 : c);
    }
  } else {
    for (int d = 0; d < 3; ++d) {
      int c = (int)((x[d] - g.origin[d]) / g.h[d]);
      ci[d] = c < 0 ? 0 : (c >= g.nc[d] ? g.nc[d] - 1 : c);
      w.wpos[3 * a + d] = x[d];
      w.wrap[3 * a + d] = 0;
    }
  }
  int cell = (ci[0] * g.nc[1] + ci[1]) * g.nc[2] + ci[2];
  w.cell_of[a] = cell;
  atomicAdd(&w.cell_count[cell], 1);
}

// Exclusive scan of cell_count into cell_start by one block; cell_count becomes
// the scatter cursor (zeroed).
__global__ void k_cell_scan(Work w, const Grid* __restrict__ gp) {
  __shared__ int part[1024];
  const Grid& g = *gp;
  int n = g.nc[0] * g.nc[1] * g.nc[2];
  int per = (n + blockDim.x - 1) / blockDim.x;
  int b = threadIdx.x * per, e = min(n, b + per);
  int s = 0;
  for (int i = b; i < e; ++i) s += w.cell_count[i];
  part[threadIdx.x] = s;
  __syncthreads();
  for (int off = 1; off < (int)blockDim.x; off <<= 1) {
    int v = threadIdx.x >= off ? part[threadIdx.x - off] : 0;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  int run = part[threadIdx.x] - s;
  for (int i = b; i < e; ++i) {
    int c = w.cell_count[i];
    w.cell_start[i] = run;
    w.cell_count[i] = 0;
    run += c;
  }
  if (threadIdx.x == blockDim.x - 1) w.cell_start[n] = run;
}

__global__ void k_scatter(Work w) {
  int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= w.n_atoms) return;
  int c = w.cell_of[a];
  int slot = atomicAdd(&w.cell_count[c], 1);
  w.cell_atoms[w.cell_start[c] + slot] = a;
}

// ---------------------------------------------------------------------------------------
// site lists: one block per central atom, candidates collected in shared memory and
// bitonic-sorted by (r^2, atom, displacement)
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ bool site_less(double ra, int aa, const double* xa, double rb, int ab,
                                          const double* xb) {
  if (ra != rb) return ra < rb;
  if (aa != ab) return aa < ab;
  if (xa[0] != xb[0]) return xa[0] < xb[0];
  if (xa[1] != xb[1]) return xa[1] < xb[1];
  return xa[2] < xb[2];
}

// Displacement d (Angstrom) of the image img of atom j from the centre at wrapped position xk,
// and its square, with every operation rounded separately (no contraction): the build and the
// refresh of the site lists produce the same bits.
__device__ __forceinline__ double site_disp(const Work& w, const Grid& g, int j, const int* img, const double* xk,
                                            double* d) {
  for (int e = 0; e < 3; ++e) {
    double sh = 0.0;
    if (g.periodic)
      sh = __dadd_rn(__dadd_rn(__dmul_rn((double)img[0], g.cell[0 * 3 + e]), __dmul_rn((double)img[1], g.cell[1 * 3 + e])),
                     __dmul_rn((double)img[2], g.cell[2 * 3 + e]));
    d[e] = __dsub_rn(__dadd_rn(w.wpos[3 * j + e], sh), xk[e]);
  }
  return __dadd_rn(__dadd_rn(__dmul_rn(d[0], d[0]), __dmul_rn(d[1], d[1])), __dmul_rn(d[2], d[2]));
}

// Sort the n candidates of centre k (shared memory: key r^2, atom, displacement, image) by
// (r^2, atom, displacement) and store them with the prefix counts; overflow beyond cap was
// flagged by the caller.
__device__ void sites_sort_store(Work& w, const DevParams& p, int k, int n, int cnt, double* key, double* dx, int* at,
                                 int* im) {
  const int cap = w.site_cap;
  const bool overflow = cnt > cap;
  int P = 1;
  while (P < n) P <<= 1;
  for (int i = n + threadIdx.x; i < P; i += blockDim.x) {
    key[i] = 1e300;
    at[i] = 0x7fffffff;
    dx[3 * i] = dx[3 * i + 1] = dx[3 * i + 2] = 0.0;
    im[3 * i] = im[3 * i + 1] = im[3 * i + 2] = 0;
  }
  __syncthreads();
  for (int size = 2; size <= P; size <<= 1)
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int i = threadIdx.x; i < P / 2; i += blockDim.x) {
        int lo = 2 * i - (i & (stride - 1));
        int hi = lo + stride;
        bool up = ((lo & size) == 0);
        bool less = site_less(key[hi], at[hi], dx + 3 * hi, key[lo], at[lo], dx + 3 * lo);
        if (less == up) {
          double tk = key[lo]; key[lo] = key[hi]; key[hi] = tk;
          int ta = at[lo]; at[lo] = at[hi]; at[hi] = ta;
          for (int d = 0; d < 3; ++d) {
            double t = dx[3 * lo + d]; dx[3 * lo + d] = dx[3 * hi + d]; dx[3 * hi + d] = t;
            int ti = im[3 * lo + d]; im[3 * lo + d] = im[3 * hi + d]; im[3 * hi + d] = ti;
          }
        }
      }
      __syncthreads();
    }
  // write out and count the prefixes
  __shared__ int c1, cs, c12;
  if (threadIdx.x == 0) { c1 = 0; cs = 0; c12 = 0; }
  __syncthreads();
  long long base = (long long)k * cap;
  const double ib = 1.0 / LMBD_BOHR;
  int l1 = 0, ls = 0, l12 = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double r2 = key[i];
    const int j = at[i];
    w.site_atom[base + i] = j;
    w.site_x[3 * (base + i) + 0] = dx[3 * i + 0] * ib;
    w.site_x[3 * (base + i) + 1] = dx[3 * i + 1] * ib;
    w.site_x[3 * (base + i) + 2] = dx[3 * i + 2] * ib;
    // lattice image relative to the unwrapped positions: pos_j + n C - pos_k
    for (int d = 0; d < 3; ++d) w.site_img[3 * (base + i) + d] = im[3 * i + d] - w.wrap[3 * j + d] + w.wrap[3 * k + d];
    l1 += r2 < p.r2_scs_ang;
    ls += r2 < p.r2_sphere_ang;
    l12 += r2 < p.r2_scs2_ang;
  }
  atomicAdd(&c1, l1);
  atomicAdd(&cs, ls);
  atomicAdd(&c12, l12);
  __syncthreads();
  if (threadIdx.x == 0) {
    w.counts[k] = Counts{c1, cs, c12, n};
    // the central atom must be the unique site at distance zero (a truncated list, reported
    // as a capacity overflow, need not hold the centre)
    if (!overflow && (n < 1 || at[0] != k || key[0] != 0.0 || (n > 1 && key[1] == 0.0)))
      atomicOr(w.status, LMBD_FLAG_COINCIDENT);
  }
}

__global__ void k_sites(Work w, DevParams p, const Grid* __restrict__ gp, int c0) {
  extern __shared__ unsigned char smem[];
  const int cap = w.site_cap;                 // power of two
  double* key = (double*)smem;                // cap
  double* dx = key + cap;                     // cap x 3
  int* at = (int*)(dx + 3 * cap);             // cap
  int* im = at + cap;                         // cap x 3 image shifts of the wrapped positions
  __shared__ int cnt;
  const Grid& g = *gp;
  int k = c0 + blockIdx.x;
  if (k >= w.n_atoms) return;
  if (threadIdx.x == 0) cnt = 0;
  __syncthreads();
  double xk[3] = {w.wpos[3 * k], w.wpos[3 * k + 1], w.wpos[3 * k + 2]};
  int ck = w.cell_of[k];
  int ci[3] = {ck / (g.nc[1] * g.nc[2]), (ck / g.nc[2]) % g.nc[1], ck % g.nc[2]};
  for (int ox = -g.reach[0]; ox <= g.reach[0]; ++ox)
    for (int oy = -g.reach[1]; oy <= g.reach[1]; ++oy)
      for (int oz = -g.reach[2]; oz <= g.reach[2]; ++oz) {
        int o[3] = {ox, oy, oz};
        int cc[3], img[3];
        bool ok = true;
        for (int d = 0; d < 3; ++d) {
          int c = ci[d] + o[d];
          if (g.periodic) {
            int q = c >= 0 ? c / g.nc[d] : -((-c + g.nc[d] - 1) / g.nc[d]);
            cc[d] = c - q * g.nc[d];
            img[d] = q;
          } else {
            if (c < 0 || c >= g.nc[d]) ok = false;
            cc[d] = c;
            img[d] = 0;
          }
        }
        if (!ok) continue;
        int cell = (cc[0] * g.nc[1] + cc[1]) * g.nc[2] + cc[2];
        int b = w.cell_start[cell], e = w.cell_start[cell + 1];
        for (int t = b + threadIdx.x; t < e; t += blockDim.x) {
          int j = w.cell_atoms[t];
          double d[3];
          const double r2 = site_disp(w, g, j, img, xk, d);
          if (r2 < p.r2_list_ang) {
            int slot = atomicAdd(&cnt, 1);
            if (slot < cap) {
              key[slot] = r2;
              at[slot] = j;
              dx[3 * slot + 0] = d[0];
              dx[3 * slot + 1] = d[1];
              dx[3 * slot + 2] = d[2];
              im[3 * slot + 0] = img[0];
              im[3 * slot + 1] = img[1];
              im[3 * slot + 2] = img[2];
            }
          }
        }
      }
  __syncthreads();
  int n = cnt;
  if (n > cap) {
    if (threadIdx.x == 0) atomicOr(w.status, LMBD_FLAG_CAPACITY);
    n = cap;
  }
  sites_sort_store(w, p, k, n, cnt, key, dx, at, im);
}

// Refresh of resident site lists (trajectory frames within half a Verlet skin of the frame the
// lists were built for): every stored candidate, an atom and its lattice image relative to the
// unwrapped positions, gets its displacement recomputed from the current positions with the
// build's arithmetic, and the candidates are sorted and counted again.  The candidates hold
// every site within the list radius + skin of the build frame, so every site now within the
// list radius; the sites within it come out in the order, and with the bits, of a fresh build.
__global__ void k_sites_refresh(Work w, DevParams p, const Grid* __restrict__ gp) {
  extern __shared__ unsigned char smem[];
  const int cap = w.site_cap;
  double* key = (double*)smem;
  double* dx = key + cap;
  int* at = (int*)(dx + 3 * cap);
  int* im = at + cap;
  const Grid& g = *gp;
  const int k = blockIdx.x;
  if (k >= w.n_atoms) return;
  const int n = w.counts[k].nt;
  const long long base = (long long)k * cap;
  const double xk[3] = {w.wpos[3 * k], w.wpos[3 * k + 1], w.wpos[3 * k + 2]};
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const int j = w.site_atom[base + i];
    int img[3];
    for (int d = 0; d < 3; ++d) img[d] = w.site_img[3 * (base + i) + d] + w.wrap[3 * j + d] - w.wrap[3 * k + d];
    double d3[3];
    key[i] = site_disp(w, g, j, img, xk, d3);
    at[i] = j;
    for (int d = 0; d < 3; ++d) {
      dx[3 * i + d] = d3[d];
      im[3 * i + d] = img[d];
    }
  }
  __syncthreads();
  sites_sort_store(w, p, k, n, n, key, dx, at, im);
}

// Largest displacement of any atom from the reference frame, and a species change: flag 1 if
// some atom moved by half the skin or more (or changed species).
__global__ void k_skin_check(Work w, const double* __restrict__ ref_pos, const int* __restrict__ ref_spec,
                             double half_skin2, int* flag) {
  int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= w.n_atoms) return;
  double d2 = 0.0;
  for (int d = 0; d < 3; ++d) {
    const double t = w.pos[3 * a + d] - ref_pos[3 * a + d];
    d2 += t * t;
  }
  if (!(d2 < half_skin2) || w.species[a] != ref_spec[a]) atomicOr(flag, 1);
}

void launch_skin_check(const Work& w, const double* ref_pos, const int* ref_spec, double half_skin2, int* flag,
                       cudaStream_t s) {
  if (w.n_atoms == 0) return;
  k_skin_check<<<(w.n_atoms + 127) / 128, 128, 0, s>>>(w, ref_pos, ref_spec, half_skin2, flag);
}

void launch_sites_refresh(const Work& w, const DevParams& p, const Grid& g, cudaStream_t s, int* launches) {
  if (w.n_atoms == 0) return;
  Grid* gdev = w.grid;
  cudaMemcpyAsync(gdev, &g, sizeof(Grid), cudaMemcpyHostToDevice, s);
  k_wrap<<<(w.n_atoms + 127) / 128, 128, 0, s>>>(w, gdev);
  const size_t sm = (size_t)w.site_cap * (8 + 24 + 4 + 12);
  raise_smem_limit((const void*)k_sites_refresh, sm);
  k_sites_refresh<<<w.n_atoms, 256, sm, s>>>(w, p, gdev);
  *launches += 2;
}

void launch_neighbors(const Work& w, const DevParams& p, const Grid& g, cudaStream_t s, int* launches) {
  if (w.n_atoms == 0) return;
  Grid* gdev = w.grid;
  cudaMemcpyAsync(gdev, &g, sizeof(Grid), cudaMemcpyHostToDevice, s);
  if (!g.periodic) {
    k_bbox<<<1, 256, 0, s>>>(w, gdev, sqrt(p.r2_list_ang));
    ++*launches;
  }
  cudaMemsetAsync(w.cell_count, 0, sizeof(int) * w.ncells, s);
  int nb = (w.n_atoms + 127) / 128;
  k_bin<<<nb, 128, 0, s>>>(w, gdev);
  k_cell_scan<<<1, 1024, 0, s>>>(w, gdev);
  k_scatter<<<nb, 128, 0, s>>>(w);
  size_t sm = (size_t)w.site_cap * (8 + 24 + 4 + 12);
  raise_smem_limit((const void*)k_sites, sm);
  k_sites<<<w.n_atoms, 256, sm, s>>>(w, p, gdev, 0);
  *launches += 4;
}

// ---------------------------------------------------------------------------------------
// per-centre offsets into the variable-size workspaces (one block, 64-bit scans)
// totals: [0] sum n1, [1] sum ns, [2] sum nq N1(N1+1)/2 (packed factors, N1 = 3 n1),
//         [3] sum (3 ns)^2, [4] max n1, [5] max ns, [6] max n12, [7] sum nt,
//         [8] sum of SCS pairs, [9] sum of SCS adjacency entries, [10] max pairs,
//         [11] max coupled T_LR pairs (block-sparse T_LR, 0 otherwise),
//         [12] sum Mpad Kpad, [13] sum Mpad, [14] sum Kpad, [15] sum ns16 (sliced products)
// ---------------------------------------------------------------------------------------
#define OFF_T 256
__global__ void k_offsets(Work w, int nq) {
  __shared__ long long part[11][OFF_T];
  __shared__ int mx[5][OFF_T];
  __shared__ long long tot_nt[OFF_T];
  int N = w.n_atoms;
  int per = (N + blockDim.x - 1) / blockDim.x;
  int b = threadIdx.x * per, e = min(N, b + per);
  long long s[11] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  int m[5] = {0, 0, 0, 0, 0};
  long long snt = 0;
  for (int i = b; i < e; ++i) {
    Counts c = w.counts[i];
    long long N1 = 3LL * c.n1;
    int np = w.pcount ? w.pcount[2 * i] : 0, na = w.pcount ? w.pcount[2 * i + 1] : 0;
    s[0] += c.n1;
    s[1] += c.ns;
    s[2] += (long long)nq * N1 * (N1 + 1) / 2;
    s[3] += 9LL * c.ns * c.ns;
    s[4] += np;
    s[5] += na;
    const long long Nn = 3LL * c.ns, Mp = (Nn + 63) / 64 * 64, Kp = (Nn + 15) / 16 * 16;
    s[6] += Mp * Kp;
    s[7] += Mp;
    s[8] += Kp;
    s[9] += (c.ns + 15) / 16 * 16;
    const int spn = w.sp_np ? w.sp_np[i] : 0;
    s[10] += spn;
    m[4] = max(m[4], spn);
    m[0] = max(m[0], c.n1);
    m[1] = max(m[1], c.ns);
    m[2] = max(m[2], c.n12);
    m[3] = max(m[3], np);
    snt += c.nt;
  }
  for (int t = 0; t < 11; ++t) part[t][threadIdx.x] = s[t];
  for (int t = 0; t < 5; ++t) mx[t][threadIdx.x] = m[t];
  tot_nt[threadIdx.x] = snt;
  __syncthreads();
  for (int off = 1; off < (int)blockDim.x; off <<= 1) {
    long long v[11];
    for (int t = 0; t < 11; ++t) v[t] = threadIdx.x >= off ? part[t][threadIdx.x - off] : 0;
    __syncthreads();
    for (int t = 0; t < 11; ++t) part[t][threadIdx.x] += v[t];
    __syncthreads();
  }
  long long run[11];
  for (int t = 0; t < 11; ++t) run[t] = part[t][threadIdx.x] - s[t];
  for (int i = b; i < e; ++i) {
    Counts c = w.counts[i];
    long long N1 = 3LL * c.n1;
    w.off_k1[i] = run[0];
    w.off_s[i] = run[1];
    w.off_b[i] = run[2];
    w.off_t[i] = run[3];
    if (w.off_p) w.off_p[i] = run[4];
    if (w.off_a) w.off_a[i] = run[5];
    if (w.off_np) w.off_np[i] = run[10];
    if (w.off_tq) {
      w.off_tq[i] = run[6];
      w.off_tr[i] = run[7];
      w.off_kp[i] = run[8];
      w.off_sp[i] = run[9];
    }
    const long long Nn = 3LL * c.ns, Mp = (Nn + 63) / 64 * 64, Kp = (Nn + 15) / 16 * 16;
    run[6] += Mp * Kp;
    run[7] += Mp;
    run[8] += Kp;
    run[9] += (c.ns + 15) / 16 * 16;
    run[0] += c.n1;
    run[1] += c.ns;
    run[2] += (long long)nq * N1 * (N1 + 1) / 2;
    run[3] += 9LL * c.ns * c.ns;
    run[4] += w.pcount ? w.pcount[2 * i] : 0;
    run[5] += w.pcount ? w.pcount[2 * i + 1] : 0;
    run[10] += w.sp_np ? w.sp_np[i] : 0;
  }
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st) {
      for (int t = 0; t < 5; ++t) mx[t][threadIdx.x] = max(mx[t][threadIdx.x], mx[t][threadIdx.x + st]);
      tot_nt[threadIdx.x] += tot_nt[threadIdx.x + st];
    }
    __syncthreads();
  }
  if (threadIdx.x == blockDim.x - 1) {
    w.off_k1[N] = part[0][threadIdx.x];
    w.off_s[N] = part[1][threadIdx.x];
    w.off_b[N] = part[2][threadIdx.x];
    w.off_t[N] = part[3][threadIdx.x];
    if (w.off_p) w.off_p[N] = part[4][threadIdx.x];
    if (w.off_a) w.off_a[N] = part[5][threadIdx.x];
    if (w.off_np) w.off_np[N] = part[10][threadIdx.x];
    for (int t = 0; t < 4; ++t) w.totals[t] = part[t][threadIdx.x];
    w.totals[8] = part[4][threadIdx.x];
    w.totals[9] = part[5][threadIdx.x];
    for (int t = 6; t < 10; ++t) w.totals[6 + t] = part[t][threadIdx.x];
    if (w.off_tq) {
      w.off_tq[N] = part[6][threadIdx.x];
      w.off_tr[N] = part[7][threadIdx.x];
      w.off_kp[N] = part[8][threadIdx.x];
      w.off_sp[N] = part[9][threadIdx.x];
    }
  }
  if (threadIdx.x == 0) {
    w.totals[4] = mx[0][0];
    w.totals[5] = mx[1][0];
    w.totals[6] = mx[2][0];
    w.totals[7] = tot_nt[0];
    w.totals[10] = mx[3][0];
    w.totals[11] = mx[4][0];
  }
}

void launch_offsets(const Work& w, const DevParams& p, cudaStream_t s) {
  if (w.n_atoms == 0) return;
  k_offsets<<<1, OFF_T, 0, s>>>(w, p.nqs);
}
