// Decomposition build on the GPU (Section II-B and the sorting of Section II-C):
// ingest and support radii, Morton keys, LSD radix sort, cell tree with the
// split rule, self/pair interaction lists with recursive splitting, particle
// offsets relative to their cell, and the per-cell sorted projections along
// the 13 cell-pair axes.
#include "sph_engine.h"

#include <cfloat>

namespace sph {

// ============================================================== ingest
// Validate the inputs, compute H = gamma_K * h (rounded once to FP32) and the
// per-box extremes of H.  bid[p] is the box of input particle p.
__global__ void k_ingest(long long N, const int* __restrict__ bid, BoxDesc* box, const double* __restrict__ x,
                         const float* __restrict__ v, const float* __restrict__ m, const float* __restrict__ u,
                         const float* __restrict__ h, float gamma_k, float* __restrict__ H_out) {
  pdl_wait();
  const long long stride = (long long)gridDim.x * blockDim.x;
  // a warp whose lanes all hold particles of one box keeps that box's extremes
  // across its iterations and adds them once (the same address from every warp
  // of a large box would serialise the atomics)
  int rb = -1;
  unsigned int rmx = 0u, rmn = 0xffffffffu;
  for (long long base = (long long)blockIdx.x * blockDim.x; base < N; base += stride) {
    const long long p = base + threadIdx.x;   // every lane of a warp runs every iteration
    const bool valid = p < N;
    const int b = valid ? bid[p] : -1;
    bool ok = valid;
    float H = 0.0f;
    if (valid) {
      const double L = box[b].L;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const double xk = x[3 * p + k];
        ok &= (xk >= 0.0) && (xk < L);
        ok &= isfinite(v[3 * p + k]);
      }
      const float hp = h[p];
      ok &= isfinite(hp) && hp > 0.0f && isfinite(m[p]) && m[p] > 0.0f && isfinite(u[p]) && u[p] >= 0.0f;
      H = __fmul_rn(gamma_k, hp);
      ok &= isfinite(H) && H > 0.0f;
      if (!ok) atomicOr(&box[b].err, ERR_BAD_INPUT);
      H_out[p] = ok ? H : 0.0f;
    }
    // one atomic per warp and box: lanes of the same box reduce first (H > 0, so
    // the float bit patterns order like the values)
    const unsigned int same = __match_any_sync(0xffffffffu, b);
    const unsigned int hb = ok ? __float_as_uint(H) : 0u;
    const unsigned int mx = __reduce_max_sync(same, hb);
    const unsigned int mn = __reduce_min_sync(same, ok ? hb : 0xffffffffu);
    if (same == 0xffffffffu && b >= 0) {      // the same in every lane
      if (b != rb) {
        if (rb >= 0 && (threadIdx.x & 31) == 0) {
          if (rmx) atomicMax(reinterpret_cast<unsigned int*>(&box[rb].Hmax), rmx);
          if (rmn != 0xffffffffu) atomicMin(reinterpret_cast<unsigned int*>(&box[rb].Hmin), rmn);
        }
        rb = b;
        rmx = 0u;
        rmn = 0xffffffffu;
      }
      rmx = max(rmx, mx);
      rmn = min(rmn, mn);
    } else if (valid && (threadIdx.x & 31) == __ffs(same) - 1) {
      if (mx) atomicMax(reinterpret_cast<unsigned int*>(&box[b].Hmax), mx);
      if (mn != 0xffffffffu) atomicMin(reinterpret_cast<unsigned int*>(&box[b].Hmin), mn);
    }
  }
  if (rb >= 0 && (threadIdx.x & 31) == 0) {
    if (rmx) atomicMax(reinterpret_cast<unsigned int*>(&box[rb].Hmax), rmx);
    if (rmn != 0xffffffffu) atomicMin(reinterpret_cast<unsigned int*>(&box[rb].Hmin), rmn);
  }
}

// ============================================================== captured rebuild steps
// The fields a build recomputes for every box, reset on the device (the host
// build resets them and uploads the table; the top level k stays).
__global__ void k_box_reset(int nbox, BoxDesc* box) {
  pdl_wait();
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nbox; b += gridDim.x * blockDim.x) {
    box[b].Hmax = 0.0f;
    box[b].Hmin = __int_as_float(0x7f800000);
    box[b].err = 0u;
    box[b].drift2 = 0.0f;
    box[b].drift_u = 0.0f;
  }
}

// After the ingest of a captured rebuild step: the checks of the host build on
// each box's support radii -- valid input, H_max within the box (periodic: below
// L/4) -- and the top level they give (the finest level whose edge clears H_max
// grown by the headroom, at most dc), which must be the level the graph was
// captured with (ERR_SHAPE otherwise).
__global__ void k_check_shape(int nbox, const BoxDesc* __restrict__ box, int dc, float headroom,
                              unsigned int* __restrict__ err_all) {
  pdl_wait();
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nbox; b += gridDim.x * blockDim.x) {
    const BoxDesc& d = box[b];
    if (d.err & ERR_BAD_INPUT) atomicOr(err_all, ERR_BAD_INPUT);
    const int k0 = d.periodic ? 2 : 0;
    if (!((double)d.Hmax < ldexp(d.L, -k0) - d.margin)) {
      atomicOr(err_all, ERR_H_TOO_LARGE);
      continue;
    }
    const double hr = 1.0 + (double)headroom;
    int k = k0;
    while (k + 1 <= dc && (double)d.Hmax * hr < ldexp(d.L, -(k + 1)) - d.margin) ++k;
    if (k != d.k) atomicOr(err_all, ERR_SHAPE);
  }
}

// The end of a captured build: it held when no check failed and every count fits
// its capacity (tree nodes, selfs, pairs, the empty last expansion queue, the
// task tables, the global sort's segments); the IF node of the passes follows.
__global__ void k_check_build(cudaGraphConditionalHandle ok, const unsigned int* __restrict__ err_all,
                              const int* __restrict__ t_n, int cap_nodes, const int* __restrict__ counts, int cap_self,
                              int cap_pair, int last_q, unsigned int cap_ptask, unsigned int cap_stask,
                              const unsigned long long* __restrict__ big_count, int cap_big,
                              unsigned int* __restrict__ status) {
  pdl_wait();
  const unsigned int bad = ERR_BAD_INPUT | ERR_H_TOO_LARGE | ERR_OVERFLOW | ERR_DEPTH | ERR_SHAPE;
  const bool held = (*err_all & bad) == 0u && t_n[0] <= cap_nodes && counts[0] <= cap_self && counts[1] <= cap_pair &&
                    counts[last_q] == 0 && (unsigned int)counts[6] <= cap_ptask &&
                    (unsigned int)counts[7] <= cap_stask && (long long)(*big_count >> 40) <= (long long)cap_big;
  cudaGraphSetConditional(ok, held ? 1u : 0u);
  *status = held ? 1u : 0u;
}

// ============================================================== keys
// key = box << (3 dcap) | Morton(floor((x / L) 2^dcap)) with the cell index
// clamped to [0, 2^dcap - 1]; the value is the input index.
__global__ void k_keys(long long N, int dcap, const int* __restrict__ bid, const BoxDesc* __restrict__ box,
                       const double* __restrict__ x, unsigned long long* __restrict__ key,
                       unsigned int* __restrict__ val) {
  pdl_wait();
  const double scale = ldexp(1.0, dcap);
  const unsigned int qmax = (1u << dcap) - 1u;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < N; p += (long long)gridDim.x * blockDim.x) {
    const int b = bid[p];
    const double L = box[b].L;
    unsigned int q[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const double uu = box[b].pow2 ? x[3 * p + k] * box[b].invL : __ddiv_rn(x[3 * p + k], L);
      double f = floor(__dmul_rn(uu, scale));
      f = fmin(fmax(f, 0.0), (double)qmax);
      q[k] = (unsigned int)f;
    }
    key[p] = ((unsigned long long)b << (3 * dcap)) | morton3(q[0], q[1], q[2]);
    val[p] = (unsigned int)p;
  }
}

// box of every particle from the box offsets (off[0..nbox], off[nbox] = N)
__global__ void k_box_ids(long long N, int nbox, const long long* __restrict__ off, int* __restrict__ bid) {
  pdl_wait();
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < N; p += (long long)gridDim.x * blockDim.x) {
    int lo = 0, hi = nbox - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (off[mid] <= p) lo = mid;
      else hi = mid - 1;
    }
    bid[p] = lo;
  }
}

// Moves of input-order state for a new box layout: block row y moves
// tab[3y + 2] particles from offset tab[3y + 1] to offset tab[3y].
__global__ void k_relayout(const long long* __restrict__ tab, const double* __restrict__ x,
                           const float* __restrict__ v, const float* __restrict__ m, const float* __restrict__ u,
                           const float* __restrict__ h, const float4* __restrict__ hh, const float4* __restrict__ a,
                           double* __restrict__ nx, float* __restrict__ nv, float* __restrict__ nm,
                           float* __restrict__ nu, float* __restrict__ nh, float4* __restrict__ nhh,
                           float4* __restrict__ na) {
  pdl_wait();
  const long long dst = tab[3 * blockIdx.y], src = tab[3 * blockIdx.y + 1], n = tab[3 * blockIdx.y + 2];
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
    const long long s = src + q, d = dst + q;
    nx[3 * d] = x[3 * s];
    nx[3 * d + 1] = x[3 * s + 1];
    nx[3 * d + 2] = x[3 * s + 2];
    nv[3 * d] = v[3 * s];
    nv[3 * d + 1] = v[3 * s + 1];
    nv[3 * d + 2] = v[3 * s + 2];
    nm[d] = m[s];
    nu[d] = u[s];
    nh[d] = h[s];
    nhh[d] = hh[s];
    na[d] = a[s];
  }
}

// ============================================================== decomposition reuse
// Largest displacement of every box since its decomposition was built (FP64,
// periodic minimum image), as the bits of a non-negative double (they order
// like the values).
__global__ void k_displacement(long long N, const int* __restrict__ bid, const BoxDesc* __restrict__ box,
                               const double* __restrict__ x, const double* __restrict__ xb,
                               unsigned long long* __restrict__ dmax) {
  pdl_wait();
  const long long stride = (long long)gridDim.x * blockDim.x;
  // a warp whose lanes all hold particles of one box keeps that box's largest
  // displacement across its iterations and adds it once (see k_ingest)
  int rb = -1;
  unsigned long long rbits = 0ull;
  for (long long base = (long long)blockIdx.x * blockDim.x; base < N; base += stride) {
    const long long p = base + threadIdx.x;   // every lane of a warp runs every iteration
    const bool valid = p < N;
    const int b = valid ? bid[p] : -1;
    double d2 = 0.0;
    if (valid) {
      const double L = box[b].L, halfL = 0.5 * box[b].L;
      const int per = box[b].periodic;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        double t = x[3 * p + k] - xb[3 * p + k];
        if (per) {
          if (t > halfL) t -= L;
          else if (t < -halfL) t += L;
        }
        d2 = fma(t, t, d2);
      }
    }
    unsigned long long bits = valid ? (unsigned long long)__double_as_longlong(sqrt(d2)) : 0ull;
    const int b0 = __shfl_sync(0xffffffffu, b, 0);
    if (__all_sync(0xffffffffu, !valid || b == b0)) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long y = __shfl_xor_sync(0xffffffffu, bits, o);
        bits = y > bits ? y : bits;
      }
      if (b0 >= 0 && __all_sync(0xffffffffu, valid)) {
        if (b0 != rb) {
          if (rb >= 0 && (threadIdx.x & 31) == 0) atomicMax(&dmax[rb], rbits);
          rb = b0;
          rbits = 0ull;
        }
        rbits = bits > rbits ? bits : rbits;
      } else if ((threadIdx.x & 31) == 0 && b0 >= 0) {
        atomicMax(&dmax[b0], bits);
      }
    } else if (valid) {
      atomicMax(&dmax[b], bits);
    }
  }
  if (rb >= 0 && (threadIdx.x & 31) == 0) atomicMax(&dmax[rb], rbits);
}

// The limit every particle's H must stay below with the decomposition kept:
// the split limits along its chain of cells minus twice its box's largest
// displacement (a pair within H may then have been up to H + 2 d apart when the
// cells were assigned).  flag = 1 when some particle's current H is not below
// its limit, i.e. the decomposition must be rebuilt.
__global__ void k_reuse_limits(long long N, int box_shift, const unsigned long long* __restrict__ key, Tree T,
                               const unsigned int* __restrict__ leaf_of, const unsigned int* __restrict__ perm,
                               const float* __restrict__ h, float gamma_k,
                               const unsigned long long* __restrict__ dmax, float* __restrict__ hlimp,
                               unsigned int* __restrict__ flag) {
  pdl_wait();
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < N; p += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(key[p] >> box_shift);
    int id = (int)leaf_of[p];
    double lim = 1e300;
    while (id >= 0) {
      lim = fmin(lim, T.hlim[id]);
      id = T.parent[id];
    }
    lim -= 2.0 * __longlong_as_double((long long)dmax[b]);
    const float lf = __double2float_rz(lim);
    hlimp[p] = lf;
    const float H = __fmul_rn(gamma_k, h[perm[p]]);
    if (!(H < lf)) atomicOr(flag, 1u);
  }
}

// Largest H of every cell from its leaves (cell H_max entries start at 0): one
// warp per leaf, then a climb that stops at the first cell already covering it.
__global__ void k_leaf_hmax(Tree T, int nnodes, const float* __restrict__ Hs) {
  pdl_wait();
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int id = warp; id < nnodes; id += nwarps) {
    if (T.child[id] >= 0) continue;
    const unsigned int s = T.start[id], c = T.count[id];
    float hm = 0.0f;
    for (unsigned int q = lane; q < c; q += 32) hm = fmaxf(hm, Hs[s + q]);
    hm = warp_max(hm);
    if (lane != 0) continue;
    for (int a = id; a >= 0; a = T.parent[a]) {
      if (T.hmax[a] >= hm) break;
      atomic_max_pos(&T.hmax[a], hm);
    }
  }
}

// Cluster boxes from the current offsets (membership kept): one warp per cluster.
__global__ void k_tile_boxes(long long ntile, Tiles TL, const float4* __restrict__ pos4) {
  pdl_wait();
  const int lane = threadIdx.x & 31;
  const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long t = warp; t < ntile; t += nwarps) {
    const unsigned int n = TL.n[t], s0 = TL.start[t];
    float4 lo = make_float4(FLT_MAX, FLT_MAX, FLT_MAX, 0.0f), hi = make_float4(-FLT_MAX, -FLT_MAX, -FLT_MAX, 0.0f);
    if ((unsigned int)lane < n) {
      const float4 a = pos4[s0 + lane];
      lo = make_float4(a.x, a.y, a.z, a.w);
      hi = make_float4(a.x, a.y, a.z, 0.0f);
    }
    lo.x = warp_min(lo.x); lo.y = warp_min(lo.y); lo.z = warp_min(lo.z); lo.w = warp_max(lo.w);
    hi.x = warp_max(hi.x); hi.y = warp_max(hi.y); hi.z = warp_max(hi.z);
    if (lane == 0) {
      TL.lo[t] = lo;
      TL.hi[t] = hi;
      TL.active[t] = 1;
    }
  }
}

// ============================================================== radix sort
// Stable LSD radix sort of (64-bit key, 32-bit value), 8-bit digits.  Each
// pass: per-tile digit histograms, one exclusive scan of the digit-major
// histogram table, then a stable scatter that ranks equal digits by
// (round, warp, lane) order inside the tile.
constexpr int RS_THREADS = 256;
constexpr int RS_ITEMS = 8;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;

__global__ void k_radix_hist(long long n, const unsigned long long* __restrict__ key, int shift,
                             unsigned int* __restrict__ hist, int ntiles) {
  pdl_wait();
  __shared__ unsigned int cnt[256];
  cnt[threadIdx.x] = 0;
  __syncthreads();
  const long long base = (long long)blockIdx.x * RS_TILE;
  for (int r = 0; r < RS_ITEMS; ++r) {
    const long long i = base + r * RS_THREADS + threadIdx.x;
    if (i < n) atomicAdd(&cnt[(unsigned int)(key[i] >> shift) & 255u], 1u);
  }
  __syncthreads();
  hist[(long long)threadIdx.x * ntiles + blockIdx.x] = cnt[threadIdx.x];
}

__global__ void k_radix_scatter(long long n, const unsigned long long* __restrict__ kin,
                                const unsigned int* __restrict__ vin, unsigned long long* __restrict__ kout,
                                unsigned int* __restrict__ vout, int shift, const unsigned int* __restrict__ offs,
                                int ntiles) {
  pdl_wait();
  __shared__ unsigned int base[256];
  __shared__ unsigned int wcnt[RS_THREADS / 32][256];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  base[tid] = offs[(long long)tid * ntiles + blockIdx.x];
  for (int k = 0; k < RS_THREADS / 32; ++k) wcnt[k][tid] = 0;
  __syncthreads();
  const long long tile0 = (long long)blockIdx.x * RS_TILE;
  const unsigned int lt = (1u << lane) - 1u;
  for (int r = 0; r < RS_ITEMS; ++r) {
    const long long i = tile0 + r * RS_THREADS + tid;
    const bool valid = i < n;
    unsigned long long k = valid ? kin[i] : 0ull;
    const unsigned int d = valid ? ((unsigned int)(k >> shift) & 255u) : 256u;
    const unsigned int peers = __match_any_sync(0xffffffffu, d);
    const unsigned int lrank = __popc(peers & lt);
    if (valid && lrank == 0) wcnt[w][d] = __popc(peers);
    __syncthreads();
    if (valid) {
      unsigned int pre = 0;
      for (int q = 0; q < w; ++q) pre += wcnt[q][d];
      const unsigned int pos = base[d] + pre + lrank;
      kout[pos] = k;
      vout[pos] = vin[i];
    }
    __syncthreads();
    unsigned int tot = 0;
    for (int q = 0; q < RS_THREADS / 32; ++q) {
      tot += wcnt[q][tid];
      wcnt[q][tid] = 0;
    }
    base[tid] += tot;
    __syncthreads();
  }
}

// ---------------------------------------------------------- exclusive scan (u32)
constexpr int SC_THREADS = 256;
constexpr int SC_ITEMS = 8;
constexpr int SC_TILE = SC_THREADS * SC_ITEMS;

__device__ unsigned int block_exclusive_scan(unsigned int v, unsigned int* tmp, unsigned int& total) {
  // tmp: 32 words of shared memory
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  unsigned int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) tmp[w] = x;
  __syncthreads();
  if (w == 0) {
    const int nw = blockDim.x >> 5;
    unsigned int s = lane < nw ? tmp[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned int y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < nw) tmp[lane] = s;
  }
  __syncthreads();
  const unsigned int before = (w > 0 ? tmp[w - 1] : 0u) + x - v;
  total = tmp[(blockDim.x >> 5) - 1];
  __syncthreads();
  return before;
}

// A scan may take its length from the device (n_dev: *n_dev + 1 entries, at most
// n) and run only in the later passes of an h iteration (gate: the iteration
// counter, which the kernels read; the scan is skipped in a first or stopped pass).
__device__ __forceinline__ bool scan_len(long long& n, const unsigned int* n_dev, const int* gate) {
  if (gate && !(gate[0] > 1 && gate[2] == 0)) return false;
  if (n_dev) n = min(n, (long long)*n_dev + 1);
  return true;
}

// in and out may be the same array: every thread reads its items before writing them
__global__ void k_scan_tiles(long long n, const unsigned int* in, unsigned int* out,
                             unsigned int* __restrict__ tile_sums, const unsigned int* __restrict__ n_dev,
                             const int* __restrict__ gate) {
  pdl_wait();
  if (!scan_len(n, n_dev, gate) || (long long)blockIdx.x * SC_TILE >= n) return;
  __shared__ unsigned int tmp[32];
  const long long base = (long long)blockIdx.x * SC_TILE + (long long)threadIdx.x * SC_ITEMS;
  unsigned int loc[SC_ITEMS];
  unsigned int s = 0;
#pragma unroll
  for (int k = 0; k < SC_ITEMS; ++k) {
    loc[k] = (base + k < n) ? in[base + k] : 0u;
    s += loc[k];
  }
  unsigned int total;
  unsigned int run = block_exclusive_scan(s, tmp, total);
#pragma unroll
  for (int k = 0; k < SC_ITEMS; ++k) {
    if (base + k < n) out[base + k] = run;
    run += loc[k];
  }
  if (threadIdx.x == 0) tile_sums[blockIdx.x] = total;
}

// single block: exclusive scan of the tile sums in place (any count), total -> *total
__global__ void k_scan_sums(int ntiles, unsigned int* __restrict__ sums, unsigned int* __restrict__ total_out,
                            long long n, const unsigned int* __restrict__ n_dev, const int* __restrict__ gate) {
  pdl_wait();
  if (!scan_len(n, n_dev, gate)) return;
  ntiles = min(ntiles, (int)((n + SC_TILE - 1) / SC_TILE));
  __shared__ unsigned int tmp[32];
  unsigned int carry = 0;
  for (int base = 0; base < ntiles; base += blockDim.x) {
    const int i = base + threadIdx.x;
    const unsigned int v = i < ntiles ? sums[i] : 0u;
    unsigned int total;
    const unsigned int ex = block_exclusive_scan(v, tmp, total);
    if (i < ntiles) sums[i] = carry + ex;
    carry += total;
  }
  if (threadIdx.x == 0 && total_out) *total_out = carry;
}

__global__ void k_scan_add(long long n, unsigned int* __restrict__ out, const unsigned int* __restrict__ sums,
                           const unsigned int* __restrict__ n_dev, const int* __restrict__ gate) {
  pdl_wait();
  if (!scan_len(n, n_dev, gate) || (long long)blockIdx.x * SC_TILE >= n) return;
  const long long base = (long long)blockIdx.x * SC_TILE + (long long)threadIdx.x * SC_ITEMS;
  const unsigned int add = sums[blockIdx.x];
#pragma unroll
  for (int k = 0; k < SC_ITEMS; ++k)
    if (base + k < n) out[base + k] += add;
}

void exclusive_scan(const unsigned int* in, unsigned int* out, long long n, unsigned int* tile_sums,
                    unsigned int* total, cudaStream_t st, const unsigned int* n_dev, const int* gate) {
  const long long ntiles = (n + SC_TILE - 1) / SC_TILE;
  if (ntiles == 0) return;
  launch_pdl(k_scan_tiles, (unsigned)ntiles, SC_THREADS, st, n, in, out, tile_sums, n_dev, gate); count_launch();
  launch_pdl(k_scan_sums, 1, 1024, st, (int)ntiles, tile_sums, total, n, n_dev, gate); count_launch();
  launch_pdl(k_scan_add, (unsigned)ntiles, SC_THREADS, st, n, out, tile_sums, n_dev, gate); count_launch();
}

long long radix_scratch_words(long long n) {
  const long long ntiles = (n + RS_TILE - 1) / RS_TILE;
  return 256 * ntiles + (256 * ntiles + SC_TILE - 1) / SC_TILE + 16;
}

// Sorts (k0, v0) by the low `bits` bits of the key; the result lands in
// (k0, v0) (using (k1, v1) as the other half of each pass).
void radix_sort(unsigned long long* k0, unsigned int* v0, unsigned long long* k1, unsigned int* v1, long long n,
                int bits, unsigned int* scratch, cudaStream_t st) {
  if (n <= 1 || bits <= 0) return;
  const long long ntiles = (n + RS_TILE - 1) / RS_TILE;
  unsigned int* hist = scratch;
  unsigned int* sums = scratch + 256 * ntiles;
  int passes = (bits + 7) / 8;
  unsigned long long *ka = k0, *kb = k1;
  unsigned int *va = v0, *vb = v1;
  for (int p = 0; p < passes; ++p) {
    const int shift = 8 * p;
    launch_pdl(k_radix_hist, (unsigned)ntiles, RS_THREADS, st, n, ka, shift, hist, (int)ntiles); count_launch();
    exclusive_scan(hist, hist, 256 * ntiles, sums, nullptr, st);
    launch_pdl(k_radix_scatter, (unsigned)ntiles, RS_THREADS, st, n, ka, va, kb, vb, shift, hist, (int)ntiles); count_launch();
    std::swap(ka, kb);
    std::swap(va, vb);
  }
  if (ka != k0) {
    cudaMemcpyAsync(k0, ka, n * sizeof(unsigned long long), cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(v0, va, n * sizeof(unsigned int), cudaMemcpyDeviceToDevice, st);
  }
}

// ============================================================== gather
// H, velocity and u in key order.  Inside a kick-drift-kick step (vpred = 1) the
// passes see v and u predicted to the end of the step with the previous forces,
// v_{n+1/2} + a_n dt/2 and u_{n+1/2} + (du/dt)_n dt/2, so that the velocity- and
// u-dependent terms of the force pass are taken at the time of the positions.
__global__ void k_gather_sorted(long long N, const unsigned int* __restrict__ perm, const float* __restrict__ H_in,
                                const float* __restrict__ v, const float* __restrict__ u, const int* __restrict__ bid,
                                const BoxDesc* __restrict__ box, const float4* __restrict__ a_in, int vpred,
                                float* __restrict__ Hs, float4* __restrict__ vel4) {
  pdl_wait();
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < N; p += (long long)gridDim.x * blockDim.x) {
    const unsigned int i = perm[p];
    Hs[p] = H_in[i];
    float4 w = make_float4(v[3ll * i], v[3ll * i + 1], v[3ll * i + 2], u[i]);
    if (vpred) {
      const float hdt = (float)(0.5 * box[bid[i]].dt);
      if (hdt != 0.0f) {
        const float4 a = a_in[i];
        w.x += a.x * hdt;
        w.y += a.y * hdt;
        w.z += a.z * hdt;
        w.w = fmaxf(w.w + a.w * hdt, 0.0f);
      }
    }
    vel4[p] = w;
  }
}

// ============================================================== cell tree
__device__ __forceinline__ unsigned long long prefix_at(unsigned long long key, int dcap, int level, int box_shift) {
  // box bits stay on top of the prefix
  const unsigned long long box = key >> box_shift;
  const unsigned long long mort = key & ((box_shift >= 64) ? ~0ull : ((1ull << box_shift) - 1ull));
  return (box << (3 * level)) | (mort >> (3 * (dcap - level)));
}

// first index in [lo, hi) whose prefix at `level` is >= target
__device__ __forceinline__ long long lower_bound_prefix(const unsigned long long* key, long long lo, long long hi,
                                                        unsigned long long target, int dcap, int level,
                                                        int box_shift) {
  while (lo < hi) {
    const long long mid = (lo + hi) >> 1;
    if (prefix_at(key[mid], dcap, level, box_shift) < target) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// Integer coordinates of a cell from its prefix (box bits removed).
__device__ __forceinline__ void cell_coords(unsigned long long prefix, int level, unsigned int& cx, unsigned int& cy,
                                            unsigned int& cz) {
  const unsigned long long mort = level > 0 ? (prefix & ((1ull << (3 * level)) - 1ull)) : 0ull;
  cx = compact3(mort);
  cy = compact3(mort >> 1);
  cz = compact3(mort >> 2);
}

__global__ void k_top_nodes(long long N, int dcap, int box_shift, const BoxDesc* __restrict__ box,
                            const unsigned long long* __restrict__ key, Tree T, int cap_nodes,
                            int* __restrict__ top_at, unsigned int* __restrict__ err_all) {
  pdl_wait();
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < N; p += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(key[p] >> box_shift);
    const BoxDesc bd = box[b];
    const unsigned long long pre = prefix_at(key[p], dcap, bd.k, box_shift);
    const bool start = (p == bd.off) || (prefix_at(key[p - 1], dcap, bd.k, box_shift) != pre);
    if (!start) continue;
    const int id = atomicAdd(&T.n_nodes[0], 1);
    if (id >= cap_nodes) {
      atomicOr(err_all, ERR_OVERFLOW);
      continue;
    }
    const long long end = lower_bound_prefix(key, p, bd.off + bd.n, pre + 1, dcap, bd.k, box_shift);
    T.start[id] = (unsigned int)p;
    T.count[id] = (unsigned int)(end - p);
    T.key[id] = pre;
    T.level[id] = bd.k;
    T.box[id] = b;
    T.parent[id] = -1;
    T.child[id] = -1;
    T.nchild[id] = 0;
    top_at[p] = id;
  }
}

// One round of the cell tree, one block of TREE_THREADS per large frontier node
// (a top cell can hold a large share of the box) and one warp per small one: the
// node's statistics and the
// split rule of Section II-B / III-B -- split iff level < dcap,
// count > leaf_max and n_small > split_frac * count, with
// n_small = #{H < edge/2 - margin} -- and, for a split node, its children: the
// non-empty octants, counted from the Morton digit of the next level in the
// same pass over the node's particles (sorted keys make each octant a
// contiguous range).  Children of one node get consecutive ids.  capped: dcap is
// a bound below the full depth (the previous build's depth plus one); a node at
// dcap that the rule would split sets ERR_DEPTH, and the build is redone at the
// full depth.  The deepest level of any node goes to n_nodes[5].
constexpr int TREE_THREADS = 256;

// k consecutive node ids from one atomic (a compare-and-swap loop serialised the
// thousands of nodes that split in one round).  When they do not all fit under
// the capacity, the ids that do are written as empty nodes (no particles, no
// children), so that every id below the capacity is a valid node for the rest of
// the build, which the overflow flag then redoes with more room; -1 then.
__device__ __forceinline__ int alloc_nodes(Tree& T, int k, int cap, int level, int box) {
  const int old = atomicAdd(&T.n_nodes[0], k);
  if (old + k <= cap) return old;
  for (int i = old; i < min(old + k, cap); ++i) {
    T.start[i] = 0;
    T.count[i] = 0;
    T.key[i] = 0ull;
    T.level[i] = level;
    T.box[i] = box;
    T.parent[i] = -1;
    T.child[i] = -1;
    T.nchild[i] = 0;
  }
  return -1;
}

// The split decision and the writes of one node, by one warp, from its largest
// H (hm), its particles with H < edge/2 - margin (ns) and, on lane k < 8, the
// particles in octant k (mine).
__device__ __forceinline__ void tree_node_finish(Tree& T, int id, int d, const BoxDesc& bd, unsigned int s,
                                                 unsigned int c, bool may_split, float hm, unsigned int ns,
                                                 unsigned int mine, int dcap, int leaf_max, float split_frac,
                                                 int capped, int cap_nodes, unsigned int* __restrict__ err_all) {
  const int lane = threadIdx.x & 31;
  const bool sp = may_split && (double)ns > (double)split_frac * (double)c;
  const unsigned int ne = __ballot_sync(0xffffffffu, lane < 8 && mine != 0);
  const int nch = __popc(ne);
  // start of octant `lane`: the counts of the octants before it
  unsigned int before = mine;
#pragma unroll
  for (int o = 1; o < 8; o <<= 1) {
    const unsigned int y = __shfl_up_sync(0xffffffffu, before, o);
    if (lane >= o) before += y;
  }
  before -= mine;
  int c0 = -1;
  if (sp && lane == 0) c0 = alloc_nodes(T, nch, cap_nodes, d + 1, T.box[id]);
  c0 = __shfl_sync(0xffffffffu, c0, 0);
  const bool fits = c0 >= 0;
  if (sp && fits && lane < 8 && mine != 0) {
    const int cid = c0 + __popc(ne & ((1u << lane) - 1u));
    T.start[cid] = s + before;
    T.count[cid] = mine;
    T.key[cid] = (T.key[id] << 3) | (unsigned long long)lane;
    T.level[cid] = d + 1;
    T.box[cid] = T.box[id];
    T.parent[cid] = id;
    T.child[cid] = -1;
    T.nchild[cid] = 0;
  }
  if (lane == 0) {
    if (sp && !fits) atomicOr(err_all, ERR_OVERFLOW);
    if (capped && d >= dcap && (int)c > leaf_max && (double)ns > (double)split_frac * (double)c)
      atomicOr(err_all, ERR_DEPTH);
    atomicMax(&T.n_nodes[5], d);
    T.hmax[id] = hm;
    T.nsmall[id] = ns;
    T.split[id] = (sp && fits) ? 1 : 0;
    T.child[id] = (sp && fits) ? c0 : -1;
    T.nchild[id] = (sp && fits) ? nch : 0;
    T.axes[id] = 0;
    // limit the top grid sets on every particle: H < edge_k - margin
    T.hlim[id] = (T.parent[id] < 0) ? __dsub_rn(ldexp(bd.L, -d), bd.margin) : 1e300;
    unsigned int cx, cy, cz;
    cell_coords(T.key[id], d, cx, cy, cz);
    const double inv = ldexp(1.0, -d), invk = ldexp(1.0, -bd.k);
    const int sh = d - bd.k;
    const double tx = ((double)(cx >> sh) + 0.5) * invk, ty = ((double)(cy >> sh) + 0.5) * invk,
                 tz = ((double)(cz >> sh) + 0.5) * invk;
    T.cen[id] = make_float4((float)(((double)cx + 0.5) * inv - tx), (float)(((double)cy + 0.5) * inv - ty),
                            (float)(((double)cz + 0.5) * inv - tz), (float)inv);
  }
}

// Nodes of more than TREE_WARP_MAX particles take a block of TREE_THREADS each;
// the others one warp each (most nodes are small, and a block per node leaves
// its warps waiting at barriers on a few particles).
constexpr unsigned int TREE_WARP_MAX = 2048;

__global__ void __launch_bounds__(TREE_THREADS) k_tree_round(Tree T, const BoxDesc* __restrict__ box,
                                                             const float* __restrict__ Hs,
                                                             const unsigned long long* __restrict__ key, int dcap,
                                                             int leaf_max, float split_frac, int allow_split,
                                                             int capped, int cap_nodes,
                                                             unsigned int* __restrict__ err_all) {
  pdl_wait();
  constexpr int NW = TREE_THREADS / 32;
  __shared__ float s_hm[NW];
  __shared__ unsigned int s_ns[NW], s_oc[NW][8];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int f0 = T.n_nodes[1], f1 = min(T.n_nodes[2], T.n_nodes[0]);
  // large nodes: one block each
  for (int id = f0 + blockIdx.x; id < f1; id += gridDim.x) {
    const unsigned int c = T.count[id];
    if (c <= TREE_WARP_MAX) continue;   // the same for the whole block
    const int d = T.level[id];
    const BoxDesc bd = box[T.box[id]];
    const double half = __dsub_rn(ldexp(bd.L, -(d + 1)), bd.margin);
    const unsigned int s = T.start[id];
    const bool may_split = allow_split && d < dcap && (int)c > leaf_max;
    const int dig = 3 * (dcap - d - 1);   // Morton digit of level d + 1 (when may_split)
    float hm = 0.0f;
    unsigned int ns = 0;
    unsigned int oc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (unsigned int q = threadIdx.x; q < c; q += TREE_THREADS) {
      const float H = Hs[s + q];
      hm = fmaxf(hm, H);
      ns += ((double)H < half) ? 1u : 0u;
      if (may_split) {
        const unsigned int o = (unsigned int)(key[s + q] >> dig) & 7u;
#pragma unroll
        for (int k = 0; k < 8; ++k) oc[k] += (o == (unsigned int)k) ? 1u : 0u;
      }
    }
    hm = warp_max(hm);
    ns = __reduce_add_sync(0xffffffffu, ns);
    if (may_split) {
#pragma unroll
      for (int k = 0; k < 8; ++k) oc[k] = __reduce_add_sync(0xffffffffu, oc[k]);
    }
    if (lane == 0) {
      s_hm[w] = hm;
      s_ns[w] = ns;
#pragma unroll
      for (int k = 0; k < 8; ++k) s_oc[w][k] = oc[k];
    }
    __syncthreads();
    if (w == 0) {
      hm = lane < NW ? s_hm[lane] : 0.0f;
      ns = lane < NW ? s_ns[lane] : 0u;
      hm = warp_max(hm);
      ns = __reduce_add_sync(0xffffffffu, ns);
      // lane k < 8 holds octant k's count
      unsigned int mine = 0;
      if (lane < 8)
        for (int k = 0; k < NW; ++k) mine += s_oc[k][lane];
      tree_node_finish(T, id, d, bd, s, c, may_split, hm, ns, mine, dcap, leaf_max, split_frac, capped, cap_nodes,
                       err_all);
    }
    __syncthreads();
  }
  // the other nodes: one warp each
  for (int id = f0 + (int)(blockIdx.x * NW + w); id < f1; id += (int)(gridDim.x * NW)) {
    const unsigned int c = T.count[id];
    if (c > TREE_WARP_MAX) continue;
    const int d = T.level[id];
    const BoxDesc bd = box[T.box[id]];
    const double half = __dsub_rn(ldexp(bd.L, -(d + 1)), bd.margin);
    const unsigned int s = T.start[id];
    const bool may_split = allow_split && d < dcap && (int)c > leaf_max;
    const int dig = 3 * (dcap - d - 1);
    float hm = 0.0f;
    unsigned int ns = 0, mine = 0;
    unsigned int oc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (unsigned int q = lane; q < c; q += 32) {
      const float H = Hs[s + q];
      hm = fmaxf(hm, H);
      ns += ((double)H < half) ? 1u : 0u;
      if (may_split) {
        const unsigned int o = (unsigned int)(key[s + q] >> dig) & 7u;
#pragma unroll
        for (int k = 0; k < 8; ++k) oc[k] += (o == (unsigned int)k) ? 1u : 0u;
      }
    }
    hm = warp_max(hm);
    ns = __reduce_add_sync(0xffffffffu, ns);
    if (may_split) {
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const unsigned int t = __reduce_add_sync(0xffffffffu, oc[k]);
        if (lane == k) mine = t;
      }
    }
    tree_node_finish(T, id, d, bd, s, c, may_split, hm, ns, mine, dcap, leaf_max, split_frac, capped, cap_nodes,
                     err_all);
  }
  if (!allow_split) return;
  // the last block to finish opens the next round's frontier: the nodes this
  // round created (every block has read this round's frontier by then)
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned int done = atomicAdd(reinterpret_cast<unsigned int*>(&T.n_nodes[4]), 1u);
    if (done == gridDim.x - 1) {
      __threadfence();
      const int n0 = atomicAdd(&T.n_nodes[0], 0);
      T.n_nodes[1] = T.n_nodes[2];
      T.n_nodes[2] = min(n0, cap_nodes);
      T.n_nodes[4] = 0;
    }
  }
}

__global__ void k_frontier_init(Tree T, int cap_nodes) {
  pdl_wait();
  T.n_nodes[1] = 0;
  T.n_nodes[2] = min(T.n_nodes[0], cap_nodes);
  T.n_nodes[3] = min(T.n_nodes[0], cap_nodes);   // top cells are nodes [0, n_nodes[3])
}

// ============================================================== interaction lists
__device__ __forceinline__ void push_item(Lists Lq, int out, int kind, int a, int b, int ax, int cap_queue,
                                          unsigned int* err_all) {
  const int slot = atomicAdd(&Lq.counts[2 + out], 1);
  if (slot >= cap_queue) {
    atomicOr(err_all, ERR_OVERFLOW);
    return;
  }
  Lq.q_kind[out][slot] = kind;
  Lq.q_a[out][slot] = a;
  Lq.q_b[out][slot] = b;
  Lq.q_axis[out][slot] = ax;
}

// Top level: the self-interaction of every non-empty top cell and its pairs with
// the non-empty neighbours along the 13 positive directions (periodic images
// included; a box has at least 4 top cells per dimension when periodic).  One
// thread per (top cell, direction), each with one binary search.
__global__ void k_items_top(int ntop, Tree T, const BoxDesc* __restrict__ box, const unsigned long long* __restrict__ key,
                            const int* __restrict__ top_at, int dcap, int box_shift, Lists Lq, int cap_queue,
                            unsigned int* __restrict__ err_all) {
  pdl_wait();
  // ntop bounds the top cells, whose number the tree build left on the device
  const long long n = 13ll * min(ntop, T.n_nodes[3]);
  for (long long w = blockIdx.x * (long long)blockDim.x + threadIdx.x; w < n; w += (long long)gridDim.x * blockDim.x) {
    const int id = (int)(w / 13), a = (int)(w % 13);
    const int b = T.box[id];
    const BoxDesc bd = box[b];
    const int k = bd.k;
    if (a == 0) push_item(Lq, 0, 0, id, -1, 0, cap_queue, err_all);
    unsigned int cx, cy, cz;
    cell_coords(T.key[id], k, cx, cy, cz);
    const int side = 1 << k;
    int dx, dy, dz;
    axis_vec(a, dx, dy, dz);
    int nx = (int)cx + dx, ny = (int)cy + dy, nz = (int)cz + dz;
    if (bd.periodic) {
      nx = (nx + side) % side;
      ny = (ny + side) % side;
      nz = (nz + side) % side;
    } else if (nx < 0 || ny < 0 || nz < 0 || nx >= side || ny >= side || nz >= side) {
      continue;
    }
    const unsigned long long target = ((unsigned long long)b << (3 * k)) | morton3(nx, ny, nz);
    const long long p = lower_bound_prefix(key, bd.off, bd.off + bd.n, target, dcap, k, box_shift);
    if (p < bd.off + bd.n && prefix_at(key[p], dcap, k, box_shift) == target)
      push_item(Lq, 0, 1, id, top_at[p], a, cap_queue, err_all);
  }
}

// One round of splitting (Fig. 2): a self-interaction of a split cell becomes its
// children's selfs and the pairs between them; a pair of split cells becomes the
// adjacent child pairs across the interface iff every particle of both cells has
// H < edge/2 - margin.  Everything else is final.
// Slots for n items per lane from one counter: one atomic per warp (every lane of
// the warp calls it); returns the lane's first slot.
__device__ __forceinline__ int warp_alloc(int* counter, int n) {
  const int lane = threadIdx.x & 31;
  int incl = n;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  const int total = __shfl_sync(0xffffffffu, incl, 31);
  int base = 0;
  if (lane == 31 && total > 0) base = atomicAdd(counter, total);
  base = __shfl_sync(0xffffffffu, base, 31);
  return base + incl - n;
}

__device__ __forceinline__ void put_item(Lists Lq, int out, int slot, int kind, int a, int b, int ax, int cap_queue,
                                         unsigned int* err_all) {
  if (slot >= cap_queue) {
    atomicOr(err_all, ERR_OVERFLOW);
    return;
  }
  Lq.q_kind[out][slot] = kind;
  Lq.q_a[out][slot] = a;
  Lq.q_b[out][slot] = b;
  Lq.q_axis[out][slot] = ax;
}

// adjacent child pairs of a split pair (A, B) along axis ax: counted (emit =
// false) or written from slot on
__device__ __forceinline__ int child_pairs(const Tree& T, int A, int B, int ax, bool emit, Lists Lq, int out,
                                           int slot, int cap_queue, unsigned int* err_all) {
  int bx, by, bz;
  axis_vec(ax, bx, by, bz);
  const int ca0 = T.child[A], na = T.nchild[A], cb0 = T.child[B], nb = T.nchild[B];
  int k = 0;
  for (int i = 0; i < na; ++i) {
    const int oa = (int)(T.key[ca0 + i] & 7ull);
    for (int j = 0; j < nb; ++j) {
      const int ob = (int)(T.key[cb0 + j] & 7ull);
      const int dx = 2 * bx + (ob & 1) - (oa & 1);
      const int dy = 2 * by + ((ob >> 1) & 1) - ((oa >> 1) & 1);
      const int dz = 2 * bz + ((ob >> 2) & 1) - ((oa >> 2) & 1);
      if (abs(dx) > 1 || abs(dy) > 1 || abs(dz) > 1) continue;
      if (emit) {
        if (dir_positive(dx, dy, dz)) put_item(Lq, out, slot + k, 1, ca0 + i, cb0 + j, axis_index(dx, dy, dz), cap_queue, err_all);
        else put_item(Lq, out, slot + k, 1, cb0 + j, ca0 + i, axis_index(-dx, -dy, -dz), cap_queue, err_all);
      }
      ++k;
    }
  }
  return k;
}

// One round of splitting (Fig. 2): a self-interaction of a split cell becomes its
// children's selfs and the pairs between them; a pair of split cells becomes the
// adjacent child pairs across the interface iff every particle of both cells has
// H < edge/2 - margin.  Everything else is final.  Each lane first counts what its
// item produces, so that a warp takes its output slots with one atomic per list.
__global__ void k_items_expand(int in, Tree T, const BoxDesc* __restrict__ box, Lists Lq, int cap_queue,
                               int cap_self, int cap_pair, unsigned int* __restrict__ err_all, float headroom) {
  pdl_wait();
  const int out = in ^ 1;
  const int n = min(Lq.counts[2 + in], cap_queue);
  const int lane = threadIdx.x & 31;
  const int stride = gridDim.x * blockDim.x;
  for (int w0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31); w0 < n; w0 += stride) {
    const int it = w0 + lane;
    // what the item becomes: 0 nothing, 1 a final self, 2 a final pair, 3 split self, 4 split pair
    int what = 0, A = 0, B = 0, ax = 0, nq = 0;
    if (it < n) {
      const int kind = Lq.q_kind[in][it];
      A = Lq.q_a[in][it];
      if (kind == 0) {
        if (!T.split[A]) {
          what = 1;
        } else {
          const int nc = T.nchild[A];
          what = 3;
          nq = nc + nc * (nc - 1) / 2;
        }
      } else {
        B = Lq.q_b[in][it];
        ax = Lq.q_axis[in][it];
        const int d = T.level[A];
        const BoxDesc bd = box[T.box[A]];
        const double half = __dsub_rn(ldexp(bd.L, -(d + 1)), bd.margin);
        // split the pair when every H, grown by the headroom, stays below half the
        // edge (the interactions stay valid while H < half: that is the limit recorded)
        const double hm = (double)fmaxf(T.hmax[A], T.hmax[B]) * (1.0 + (double)headroom);
        if (!(T.split[A] && T.split[B] && hm < half)) {
          what = 2;
        } else {
          what = 4;
          atomic_min_pos(&T.hlim[A], half);
          atomic_min_pos(&T.hlim[B], half);
          nq = child_pairs(T, A, B, ax, false, Lq, out, 0, cap_queue, err_all);
        }
      }
    }
    const int s_self = warp_alloc(&Lq.counts[0], what == 1 ? 1 : 0);
    const int s_pair = warp_alloc(&Lq.counts[1], what == 2 ? 1 : 0);
    const int s_q = warp_alloc(&Lq.counts[2 + out], nq);
    if (what == 1) {
      if (s_self < cap_self) Lq.self_a[s_self] = A;
      else atomicOr(err_all, ERR_OVERFLOW);
    } else if (what == 2) {
      if (s_pair < cap_pair) {
        Lq.pair_a[s_pair] = A;
        Lq.pair_b[s_pair] = B;
        Lq.pair_axis[s_pair] = ax;
      } else {
        atomicOr(err_all, ERR_OVERFLOW);
      }
    } else if (what == 3) {
      const int c0 = T.child[A], nc = T.nchild[A];
      int k = s_q;
      for (int i = 0; i < nc; ++i) put_item(Lq, out, k++, 0, c0 + i, -1, 0, cap_queue, err_all);
      for (int i = 0; i < nc; ++i) {
        const int oi = (int)(T.key[c0 + i] & 7ull);
        for (int j = i + 1; j < nc; ++j) {
          const int oj = (int)(T.key[c0 + j] & 7ull);
          int dx = (oj & 1) - (oi & 1), dy = ((oj >> 1) & 1) - ((oi >> 1) & 1), dz = ((oj >> 2) & 1) - ((oi >> 2) & 1);
          if (dir_positive(dx, dy, dz)) put_item(Lq, out, k++, 1, c0 + i, c0 + j, axis_index(dx, dy, dz), cap_queue, err_all);
          else put_item(Lq, out, k++, 1, c0 + j, c0 + i, axis_index(-dx, -dy, -dz), cap_queue, err_all);
        }
      }
    } else if (what == 4) {
      child_pairs(T, A, B, ax, true, Lq, out, s_q, cap_queue, err_all);
    }
  }
}

// leaf of every particle, and the smallest H limit along its chain of cells
__global__ void k_leaves(Tree T, int nnodes, unsigned int* __restrict__ leaf_of) {
  pdl_wait();
  nnodes = min(nnodes, T.n_nodes[0]);   // nnodes: the capacity; the count is on the device
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int id = warp; id < nnodes; id += nwarps) {
    if (T.child[id] >= 0) continue;
    const unsigned int s = T.start[id], c = T.count[id];
    for (unsigned int q = lane; q < c; q += 32) leaf_of[s + q] = (unsigned int)id;
  }
}

__global__ void k_particle_limits(long long N, Tree T, const unsigned int* __restrict__ leaf_of,
                                  float* __restrict__ hlimp) {
  pdl_wait();
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < N; p += (long long)gridDim.x * blockDim.x) {
    int id = (int)leaf_of[p];
    double lim = 1e300;
    while (id >= 0) {
      lim = fmin(lim, T.hlim[id]);
      id = T.parent[id];
    }
    hlimp[p] = __double2float_rz(lim);
  }
}

// Particle offsets relative to the centre of their leaf (units of L, FP32) and
// the leaf centre relative to its top cell's centre (exact), plus the mass.
__global__ void k_shift(long long N, int box_shift, const unsigned long long* __restrict__ key,
                        const unsigned int* __restrict__ perm, const unsigned int* __restrict__ leaf_of, Tree T,
                        const BoxDesc* __restrict__ box, const double* __restrict__ x, const float* __restrict__ m,
                        const float* __restrict__ Hs, float4* __restrict__ pos4, float4* __restrict__ cen4) {
  pdl_wait();
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < N; p += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(key[p] >> box_shift);
    const double L = box[b].L;
    const unsigned int i = perm[p];
    const int leaf = (int)leaf_of[p];
    const int d = T.level[leaf];
    unsigned int cx, cy, cz;
    cell_coords(T.key[leaf], d, cx, cy, cz);
    const double inv = ldexp(1.0, -d);
    // x / L: a power-of-two L scales exactly, so the FP64 division is needed only otherwise
    const bool p2 = box[b].pow2 != 0;
    const double iL = box[b].invL;
    double ux = p2 ? x[3ll * i] * iL : __ddiv_rn(x[3ll * i], L);
    double uy = p2 ? x[3ll * i + 1] * iL : __ddiv_rn(x[3ll * i + 1], L);
    double uz = p2 ? x[3ll * i + 2] * iL : __ddiv_rn(x[3ll * i + 2], L);
    if (box[b].global32) {
      // plain FP32: the position is held as x / L rounded to FP32 (the offset below
      // then carries that rounding, up to 2^-25 of L per coordinate)
      ux = (double)__double2float_rn(ux);
      uy = (double)__double2float_rn(uy);
      uz = (double)__double2float_rn(uz);
    }
    double ox = ux - ((double)cx + 0.5) * inv, oy = uy - ((double)cy + 0.5) * inv, oz = uz - ((double)cz + 0.5) * inv;
    if (box[b].periodic) {
      // a particle kept in its cell after a drift across the boundary: nearest image
      ox -= rint(ox);
      oy -= rint(oy);
      oz -= rint(oz);
    }
    const float sx = (float)ox, sy = (float)oy, sz = (float)oz;
    pos4[p] = make_float4(sx, sy, sz, Hs[p]);
    const float4 c = T.cen[leaf];
    cen4[p] = make_float4(c.x, c.y, c.z, m[i]);
  }
}

// ============================================================== clusters
// Inside every leaf, put the particles whose H exceeds the leaf edge after the
// others (stable), so that warp-sized clusters hold particles of similar reach.
// lsrc[p] = the particle that moves to position p.
__global__ void k_leaf_partition(Tree T, int nnodes, const BoxDesc* __restrict__ box, const float* __restrict__ Hs,
                                 unsigned int* __restrict__ lsrc) {
  pdl_wait();
  nnodes = min(nnodes, T.n_nodes[0]);
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  const unsigned int lt = (1u << lane) - 1u;
  for (int id = warp; id < nnodes; id += nwarps) {
    if (T.child[id] >= 0) continue;
    const unsigned int s = T.start[id], c = T.count[id];
    const float thr = (float)ldexp(box[T.box[id]].L, -T.level[id]);
    unsigned int nsmall = 0;
    for (unsigned int b = 0; b < c; b += 32) {
      const unsigned int q = b + lane;
      nsmall += __popc(__ballot_sync(0xffffffffu, q < c && !(Hs[s + q] > thr)));
    }
    unsigned int os = 0, ol = nsmall;
    for (unsigned int b = 0; b < c; b += 32) {
      const unsigned int q = b + lane;
      const bool valid = q < c;
      const bool large = valid && Hs[s + q] > thr;
      const unsigned int bs = __ballot_sync(0xffffffffu, valid && !large);
      const unsigned int bl = __ballot_sync(0xffffffffu, large);
      if (valid) {
        const unsigned int dst = large ? ol + __popc(bl & lt) : os + __popc(bs & lt);
        lsrc[s + dst] = s + q;
      }
      os += __popc(bs);
      ol += __popc(bl);
    }
  }
}

__global__ void k_apply_partition(long long N, const unsigned int* __restrict__ lsrc,
                                  const unsigned int* __restrict__ perm_in, unsigned int* __restrict__ perm_out,
                                  const unsigned long long* __restrict__ key_in, unsigned long long* __restrict__ key_out,
                                  const float* __restrict__ H_in, float* __restrict__ H_out,
                                  const float4* __restrict__ vel_in, float4* __restrict__ vel_out) {
  pdl_wait();
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < N; p += (long long)gridDim.x * blockDim.x) {
    const unsigned int q = lsrc[p];
    perm_out[p] = perm_in[q];
    key_out[p] = key_in[q];
    H_out[p] = H_in[q];
    vel_out[p] = vel_in[q];
  }
}

// flag[p] = 1 where a cluster starts.  Inside each leaf, separately for its two
// H classes, the clusters are the leaves of a binary split of the class along
// its Morton keys: a node (the keys that agree on every bit from some bit b up)
// is halved at bit b - 1 while it holds more than cmax particles (the cluster
// size, at most 32: a warp's lanes).  Each cluster is then an aligned box of
// aspect ratio at most 2, much tighter than cmax particles taken in Morton order,
// which often straddle octants.  Walking a class from its first particle a, the
// next cluster is the largest node that starts at a and holds at most cmax
// particles: its bit b* is the smallest of the highest bits in which key[a]
// differs from key[a - 1] (the node must start at a) and from key[a + cmax] (it
// must end before a + cmax).  One warp per leaf.
__device__ __forceinline__ int high_bit(unsigned long long v) { return v ? 63 - __clzll((long long)v) : -1; }

__global__ void k_tile_flags(Tree T, int nnodes, int box_shift, const BoxDesc* __restrict__ box,
                             const float* __restrict__ Hs, const unsigned long long* __restrict__ key,
                             unsigned int* __restrict__ flag, int cmax) {
  pdl_wait();
  nnodes = min(nnodes, T.n_nodes[0]);
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int id = warp; id < nnodes; id += nwarps) {
    if (T.child[id] >= 0) continue;
    const unsigned int s = T.start[id], c = T.count[id];
    const float thr = (float)ldexp(box[T.box[id]].L, -T.level[id]);
    unsigned int nsmall = 0;
    for (unsigned int b = 0; b < c; b += 32) {
      const unsigned int q = b + lane;
      nsmall += __popc(__ballot_sync(0xffffffffu, q < c && !(Hs[s + q] > thr)));
    }
    const int lb = box_shift - 3 * T.level[id];      // key bits below the leaf's cell
    for (int cls = 0; cls < 2; ++cls) {
      const unsigned int beg = cls == 0 ? s : s + nsmall, end = cls == 0 ? s + nsmall : s + c;
      unsigned int a = beg;
      while (a < end) {
        const unsigned long long ka = key[a];
        int bs = lb;
        if (a > beg) bs = min(bs, high_bit(key[a - 1] ^ ka));
        if (a + cmax < end) bs = min(bs, high_bit(ka ^ key[a + cmax]));
        unsigned int n;
        if (bs < 0) {
          n = min((unsigned int)cmax, end - a);   // equal keys: no node starts here, take a chunk
        } else {
          const unsigned int q = a + 1 + lane;
          const bool in = lane < cmax - 1 && q < end && ((key[q] ^ ka) >> bs) == 0ull;
          n = 1u + __popc(__ballot_sync(0xffffffffu, in));
        }
        if ((unsigned int)lane < n) flag[a + lane] = lane == 0 ? 1u : 0u;
        a += n;
      }
    }
  }
}

// cluster table from the exclusive prefix of the flags: tile_of[p], start, size,
// leaf, box (relative to the leaf centre) and largest H
__global__ void k_tile_table(long long N, Tree T, const unsigned int* __restrict__ leaf_of,
                             const unsigned int* __restrict__ flag, const unsigned int* __restrict__ excl,
                             const float4* __restrict__ pos4, unsigned int* __restrict__ tile_of, Tiles TL,
                             int cmax) {
  pdl_wait();
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < N; p += (long long)gridDim.x * blockDim.x) {
    tile_of[p] = excl[p] + flag[p] - 1u;
    if (!flag[p]) continue;
    const unsigned int t = excl[p];
    const unsigned int leaf = leaf_of[p];
    const unsigned int end = T.start[leaf] + T.count[leaf];
    unsigned int n = 1;
    while ((unsigned int)p + n < end && n < (unsigned int)cmax && !flag[p + n]) ++n;
    float4 lo = make_float4(FLT_MAX, FLT_MAX, FLT_MAX, 0.0f);
    float4 hi = make_float4(-FLT_MAX, -FLT_MAX, -FLT_MAX, 0.0f);
    for (unsigned int q = 0; q < n; ++q) {
      const float4 a = pos4[p + q];
      lo.x = fminf(lo.x, a.x); lo.y = fminf(lo.y, a.y); lo.z = fminf(lo.z, a.z);
      hi.x = fmaxf(hi.x, a.x); hi.y = fmaxf(hi.y, a.y); hi.z = fmaxf(hi.z, a.z);
      lo.w = fmaxf(lo.w, a.w);
    }
    TL.start[t] = (unsigned int)p;
    TL.n[t] = n;
    TL.leaf[t] = leaf;
    TL.lo[t] = lo;
    TL.hi[t] = hi;
    TL.cen[t] = T.cen[leaf];
    TL.active[t] = 1;
  }
}

__global__ void k_cell_tiles(Tree T, int nnodes, const unsigned int* __restrict__ tile_of) {
  pdl_wait();
  nnodes = min(nnodes, T.n_nodes[0]);
  for (int id = blockIdx.x * blockDim.x + threadIdx.x; id < nnodes; id += gridDim.x * blockDim.x) {
    const unsigned int s = T.start[id], c = T.count[id];
    const unsigned int t0 = tile_of[s];
    T.tile0[id] = t0;
    T.ntile[id] = tile_of[s + c - 1] - t0 + 1u;
  }
}

// ============================================================== axis sorts
// Section II-C keeps, per cell, the particles sorted along each of the 13
// cell-pair axes.  Here the sorted entries are the cell's clusters, keyed by the
// lower end of the projection of their box on the axis.
__global__ void k_mark_axes(Lists Lq, int cap_pair, Tree T) {
  pdl_wait();
  const int n = min(Lq.counts[1], cap_pair);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const unsigned int bit = 1u << Lq.pair_axis[i];
    atomicOr(&T.axes[Lq.pair_a[i]], bit);
    atomicOr(&T.axes[Lq.pair_b[i]], bit);
  }
}

// Storage for the sorted lists: every (cell, needed axis) gets ntile entries.
// Cells of at most 32 clusters are not sorted: a warp tests all their clusters
// at once, so an order would end no sweep earlier (sortbase = SORT_NONE).
// Cells above SORT_SMALL clusters also list their (cell, axis) segments for the
// global sort.
// cap_entries, cap_bigent: the storage of the sorted lists and of the global
// sort's keys (a captured step; the host build passes no limit and sizes the
// storage afterwards).  A cell whose lists do not fit stays unsorted (its
// clusters are then swept in their own order) and sets ERR_OVERFLOW.
__global__ void k_sort_alloc(Tree T, int nnodes, Lists Lq, int* __restrict__ big_node, int* __restrict__ big_axis,
                             unsigned int* __restrict__ big_off, unsigned long long* __restrict__ big_count,
                             int cap_big, uint4* __restrict__ mid_seg, unsigned int* __restrict__ mid_count,
                             unsigned int cap_entries, unsigned int cap_bigent, unsigned int* __restrict__ err_all) {
  pdl_wait();
  nnodes = min(nnodes, T.n_nodes[0]);
  for (int id = blockIdx.x * blockDim.x + threadIdx.x; id < nnodes; id += gridDim.x * blockDim.x) {
    const unsigned int ax = T.axes[id];
    if (!ax) continue;
    const unsigned int c = T.ntile[id];
    if (c <= 32u) {
      T.sortbase[id] = SORT_NONE;
      continue;
    }
    const int na = __popc(ax);
    const unsigned int base = atomicAdd(reinterpret_cast<unsigned int*>(&Lq.counts[5]), (unsigned int)na * c);
    if ((unsigned long long)base + (unsigned long long)na * c > cap_entries) {
      T.sortbase[id] = SORT_NONE;
      atomicOr(err_all, ERR_OVERFLOW);
      continue;
    }
    T.sortbase[id] = base;
    atomicAdd(&Lq.counts[4], na);
    if (c <= SORT_SMALL) {
      // one shared-memory sort per (cell, axis) segment
      const unsigned int g0 = atomicAdd(mid_count, (unsigned int)na);
      unsigned int q = 0;
      for (int a = 0; a < 13; ++a) {
        if (!(ax & (1u << a))) continue;
        mid_seg[g0 + q] = make_uint4((unsigned int)id, (unsigned int)a, base + q * c, c);
        ++q;
      }
    }
    if (c > SORT_SMALL) {
      // one atomic hands out the segment numbers and their storage together, so
      // storage follows segment order (the order the global sort produces)
      const unsigned long long t =
          atomicAdd(big_count, ((unsigned long long)na << 40) | (unsigned long long)((unsigned int)na * c));
      const int s0 = (int)(t >> 40);
      const unsigned int e0 = (unsigned int)(t & ((1ull << 40) - 1ull));
      const bool fits = (unsigned long long)e0 + (unsigned long long)na * c <= cap_bigent;
      if (!fits) {
        T.sortbase[id] = SORT_NONE;    // unsorted, as above; its segments are marked empty
        atomicOr(err_all, ERR_OVERFLOW);
      }
      int q = 0;
      for (int a = 0; a < 13; ++a) {
        if (!(ax & (1u << a))) continue;
        if (s0 + q < cap_big) {
          big_node[s0 + q] = fits ? id : -1;
          big_axis[s0 + q] = a;
          big_off[s0 + q] = e0 + (unsigned int)q * c;
        }
        ++q;
      }
    }
  }
}

__device__ __forceinline__ float3 axis_unit(int a) {
  int dx, dy, dz;
  axis_vec(a, dx, dy, dz);
  const int n2 = dx * dx + dy * dy + dz * dz;
  const float s = n2 == 1 ? 1.0f : (n2 == 2 ? 0.70710678118654752f : 0.57735026918962576f);
  return make_float3(dx * s, dy * s, dz * s);
}

// lower end of the projection on u of cluster t's box, in the frame of the cell
// with centre cc (the leaf-to-cell offset is exact)
__device__ __forceinline__ float tile_rlo(const Tiles& TL, const Tree& T, unsigned int t, float4 cc, float3 u) {
  const float4 lc = TL.cen[t];
  const float4 lo = TL.lo[t], hi = TL.hi[t];
  const float ox = lc.x - cc.x, oy = lc.y - cc.y, oz = lc.z - cc.z;
  const float x = (u.x >= 0.0f ? lo.x : hi.x) + ox;
  const float y = (u.y >= 0.0f ? lo.y : hi.y) + oy;
  const float z = (u.z >= 0.0f ? lo.z : hi.z) + oz;
  return fmaf(u.x, x, fmaf(u.y, y, u.z * z));
}

// Bitonic sort of (projection, cluster) in shared memory, ordered by projection
// then cluster index: segments of more than SORT_WARP_MAX clusters (at most
// SORT_SMALL) take one CTA each, the others one warp each (a CTA on a few dozen
// clusters spends its time at barriers).
constexpr unsigned int SORT_WARP_MAX = 256;

__device__ __forceinline__ void bitonic_step(float* sr, unsigned int* si, unsigned int q, unsigned int j,
                                             unsigned int k) {
  const unsigned int l = q ^ j;
  if (l > q) {
    const bool up = (q & k) == 0;
    const float a0 = sr[q], a1 = sr[l];
    const unsigned int i0 = si[q], i1 = si[l];
    const bool gt = (a0 > a1) || (a0 == a1 && i0 > i1);
    if (gt == up) {
      sr[q] = a1; sr[l] = a0;
      si[q] = i1; si[l] = i0;
    }
  }
}

__global__ void __launch_bounds__(256) k_sort_small(const uint4* __restrict__ mid_seg,
                                                   const unsigned int* __restrict__ mid_count, Tree T, Tiles TL,
                                                   float* __restrict__ sort_r, unsigned int* __restrict__ sort_i) {
  pdl_wait();
  __shared__ float sr[SORT_SMALL];
  __shared__ unsigned int si[SORT_SMALL];
  const unsigned int nseg = *mid_count;
  for (unsigned int sg = blockIdx.x; sg < nseg; sg += gridDim.x) {
    const uint4 seg = mid_seg[sg];
    const unsigned int c = seg.w, out = seg.z;
    if (c <= SORT_WARP_MAX) continue;   // the same for the whole block
    const int id = (int)seg.x;
    unsigned int npow = 1;
    while (npow < c) npow <<= 1;
    const unsigned int t0 = T.tile0[id];
    const float4 cc = T.cen[id];
    const float3 u = axis_unit((int)seg.y);
    for (unsigned int q = threadIdx.x; q < npow; q += blockDim.x) {
      sr[q] = q < c ? tile_rlo(TL, T, t0 + q, cc, u) : FLT_MAX;
      si[q] = q;
    }
    __syncthreads();
    for (unsigned int k = 2; k <= npow; k <<= 1) {
      for (unsigned int j = k >> 1; j > 0; j >>= 1) {
        for (unsigned int q = threadIdx.x; q < npow; q += blockDim.x) bitonic_step(sr, si, q, j, k);
        __syncthreads();
      }
    }
    for (unsigned int q = threadIdx.x; q < c; q += blockDim.x) {
      sort_r[out + q] = sr[q];
      sort_i[out + q] = t0 + si[q];
    }
    __syncthreads();
  }
  // small segments: one warp each, in its own slice of the arrays
  const unsigned int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  float* wr = sr + w * SORT_WARP_MAX;
  unsigned int* wi = si + w * SORT_WARP_MAX;
  for (unsigned int sg = blockIdx.x * nw + w; sg < nseg; sg += gridDim.x * nw) {
    const uint4 seg = mid_seg[sg];
    const unsigned int c = seg.w, out = seg.z;
    if (c > SORT_WARP_MAX) continue;
    const int id = (int)seg.x;
    unsigned int npow = 1;
    while (npow < c) npow <<= 1;
    const unsigned int t0 = T.tile0[id];
    const float4 cc = T.cen[id];
    const float3 u = axis_unit((int)seg.y);
    for (unsigned int q = lane; q < npow; q += 32) {
      wr[q] = q < c ? tile_rlo(TL, T, t0 + q, cc, u) : FLT_MAX;
      wi[q] = q;
    }
    __syncwarp();
    for (unsigned int k = 2; k <= npow; k <<= 1) {
      for (unsigned int j = k >> 1; j > 0; j >>= 1) {
        for (unsigned int q = lane; q < npow; q += 32) bitonic_step(wr, wi, q, j, k);
        __syncwarp();
      }
    }
    for (unsigned int q = lane; q < c; q += 32) {
      sort_r[out + q] = wr[q];
      sort_i[out + q] = t0 + wi[q];
    }
    __syncwarp();
  }
}

// The same segments, sorted by merging instead (Section II-C: a cell's sorted list
// follows from its children's sorted lists by a merge, linear in the cell's
// clusters).  A cell's clusters are contiguous and grouped by leaf, the leaves in
// Morton order, so the cell's clusters split into runs that are its leaves (runs
// of a long leaf are cut at MERGE_RUN clusters).  Each run is ordered in place
// (rank within the run), then neighbouring runs are merged pairwise, round after
// round, up to the cell: siblings in Morton order merge first, as children into
// their parents.  An element's place in a merge is its place in its own run plus
// its rank in the partner run (binary search).  The order is by (projection,
// cluster index), the same total order the direct sort produces, so both give
// identical lists.
#define MERGE_RUN 16u
#define MERGE_ITEMS (SORT_SMALL / 256)     // consecutive clusters per thread in the scans

__device__ __forceinline__ bool key_less(float ka, unsigned int ia, float kb, unsigned int ib) {
  return ka < kb || (ka == kb && ia < ib);
}

// Exclusive scan over the 256 threads of the block (sum when MAXOP is false, max
// otherwise; identity 0).  wtot: 8 words of shared memory.
template <bool MAXOP>
__device__ __forceinline__ unsigned int block_excl_scan(unsigned int v, unsigned int* wtot) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  unsigned int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x = MAXOP ? max(x, y) : x + y;
  }
  if (lane == 31) wtot[w] = x;
  __syncthreads();
  unsigned int pre = 0;
  for (int k = 0; k < w; ++k) pre = MAXOP ? max(pre, wtot[k]) : pre + wtot[k];
  const unsigned int ex = __shfl_up_sync(0xffffffffu, x, 1);
  const unsigned int mine = lane == 0 ? 0u : ex;
  __syncthreads();
  return MAXOP ? max(pre, mine) : pre + mine;
}

__global__ void __launch_bounds__(256) k_sort_merge(const uint4* __restrict__ mid_seg,
                                                   const unsigned int* __restrict__ mid_count, Tree T, Tiles TL,
                                                   float* __restrict__ sort_r, unsigned int* __restrict__ sort_i) {
  pdl_wait();
  __shared__ float sr[2][SORT_SMALL];
  __shared__ unsigned int si[2][SORT_SMALL];         // cluster index q | run << 16
  __shared__ unsigned short rs[2][SORT_SMALL + 1];   // run starts
  __shared__ unsigned int wtot[8];
  __shared__ unsigned int s_nr;
  const unsigned int nseg = *mid_count;
  const unsigned int q0 = threadIdx.x * MERGE_ITEMS;
  for (unsigned int sg = blockIdx.x; sg < nseg; sg += gridDim.x) {
    const uint4 seg = mid_seg[sg];
    const int id = (int)seg.x;
    const unsigned int c = seg.w, out = seg.z;
    const unsigned int t0 = T.tile0[id];
    const float4 cc = T.cen[id];
    const float3 u = axis_unit((int)seg.y);
    // keys; runs start at every leaf and every MERGE_RUN clusters into a leaf:
    // the start of q's leaf is a max-scan of the leaf-start positions, the run
    // numbers a sum-scan of the run starts
    unsigned int lstart[MERGE_ITEMS];
    unsigned int m = 0;
    unsigned int prev_leaf = (q0 > 0 && q0 < c) ? TL.leaf[t0 + q0 - 1] : 0xffffffffu;
#pragma unroll
    for (int k = 0; k < (int)MERGE_ITEMS; ++k) {
      const unsigned int q = q0 + k;
      bool ls = false;
      if (q < c) {
        sr[0][q] = tile_rlo(TL, T, t0 + q, cc, u);
        const unsigned int lf = TL.leaf[t0 + q];
        ls = q == 0 || lf != prev_leaf;
        prev_leaf = lf;
      }
      if (ls) m = q;
      lstart[k] = m;          // within the thread's items; 0 when none yet
    }
    const unsigned int pm = block_excl_scan<true>(m, wtot);
    unsigned int nrun = 0;
    bool rstart[MERGE_ITEMS];
#pragma unroll
    for (int k = 0; k < (int)MERGE_ITEMS; ++k) {
      const unsigned int q = q0 + k;
      const unsigned int f = max(pm, lstart[k]);
      rstart[k] = q < c && (q - f) % MERGE_RUN == 0u;
      nrun += rstart[k] ? 1u : 0u;
    }
    unsigned int r = block_excl_scan<false>(nrun, wtot);
#pragma unroll
    for (int k = 0; k < (int)MERGE_ITEMS; ++k) {
      const unsigned int q = q0 + k;
      if (q >= c) break;
      if (rstart[k]) rs[0][r++] = (unsigned short)q;
      si[0][q] = q | ((r - 1) << 16);
    }
    if (threadIdx.x == blockDim.x - 1) s_nr = r;     // the last thread holds the total
    __syncthreads();
    unsigned int nr = s_nr;
    if (threadIdx.x == 0) rs[0][nr] = (unsigned short)c;
    __syncthreads();
    // order every run in place: rank of each element within its run
    for (unsigned int q = threadIdx.x; q < c; q += blockDim.x) {
      const unsigned int rr = si[0][q] >> 16;
      const unsigned int b = rs[0][rr], e = rs[0][rr + 1];
      const float k = sr[0][q];
      unsigned int rank = 0;
      for (unsigned int j = b; j < e; ++j) rank += key_less(sr[0][j], j, k, q) ? 1u : 0u;
      sr[1][b + rank] = k;
      si[1][b + rank] = si[0][q];
    }
    __syncthreads();
    // pairwise merges of neighbouring runs up to the whole cell; keys ping-pong
    // between buffers cur and cur ^ 1, run starts between rs[cur ^ 1] (read) and rs[cur]
    int cur = 1;
    while (nr > 1) {
      const int nxt = cur ^ 1;
      const unsigned short* rin = rs[cur ^ 1];
      for (unsigned int q = threadIdx.x; q < c; q += blockDim.x) {
        const float k = sr[cur][q];
        const unsigned int w = si[cur][q];
        const unsigned int rr = w >> 16, cq = w & 0xffffu;
        const unsigned int pr = rr ^ 1u;
        unsigned int rank = 0;
        if (pr < nr) {
          unsigned int lo = rin[pr], hi = rin[pr + 1];
          // partner elements below (k, cq)
          while (lo < hi) {
            const unsigned int mid = (lo + hi) >> 1;
            if (key_less(sr[cur][mid], si[cur][mid] & 0xffffu, k, cq)) lo = mid + 1;
            else hi = mid;
          }
          rank = lo - rin[pr];
        }
        const unsigned int dst = rin[rr & ~1u] + (q - rin[rr]) + rank;
        sr[nxt][dst] = k;
        si[nxt][dst] = cq | ((rr >> 1) << 16);
      }
      const unsigned int nn = (nr + 1) >> 1;
      for (unsigned int k2 = threadIdx.x; k2 <= nn; k2 += blockDim.x)
        rs[cur][k2] = k2 < nn ? rin[2 * k2] : (unsigned short)c;
      __syncthreads();
      nr = nn;
      cur = nxt;
    }
    for (unsigned int q = threadIdx.x; q < c; q += blockDim.x) {
      sort_r[out + q] = sr[cur][q];
      sort_i[out + q] = t0 + (si[cur][q] & 0xffffu);
    }
    __syncthreads();
  }
}

// Cells with many clusters: composite keys (segment << 32 | orderable projection)
// for one global radix sort, then scatter back into each cell's storage.
// nseg < 0: the segment count comes from the device (a captured step, capped at
// cap_big); segments marked empty (node -1) are skipped.
__global__ void k_sort_big_keys(int nseg, const int* __restrict__ big_node, const int* __restrict__ big_axis,
                                const unsigned int* __restrict__ big_off, Tree T, Tiles TL,
                                unsigned long long* __restrict__ ckey, unsigned int* __restrict__ cval,
                                const unsigned long long* __restrict__ big_count, int cap_big) {
  pdl_wait();
  if (nseg < 0) nseg = min((int)(*big_count >> 40), cap_big);
  for (int sgi = blockIdx.x; sgi < nseg; sgi += gridDim.x) {
    const int id = big_node[sgi];
    if (id < 0) continue;
    const int a = big_axis[sgi];
    const unsigned int c = T.ntile[id], t0 = T.tile0[id], o = big_off[sgi];
    const float4 cc = T.cen[id];
    const float3 u = axis_unit(a);
    for (unsigned int q = threadIdx.x; q < c; q += blockDim.x) {
      ckey[o + q] = ((unsigned long long)sgi << 32) | float_key(tile_rlo(TL, T, t0 + q, cc, u));
      cval[o + q] = q;
    }
  }
}

__global__ void k_sort_big_scatter(int nseg, const int* __restrict__ big_node, const int* __restrict__ big_axis,
                                   const unsigned int* __restrict__ big_off, Tree T, Tiles TL,
                                   const unsigned int* __restrict__ cval, float* __restrict__ sort_r,
                                   unsigned int* __restrict__ sort_i, const unsigned long long* __restrict__ big_count,
                                   int cap_big) {
  pdl_wait();
  if (nseg < 0) nseg = min((int)(*big_count >> 40), cap_big);
  for (int sgi = blockIdx.x; sgi < nseg; sgi += gridDim.x) {
    const int id = big_node[sgi];
    if (id < 0) continue;
    const int a = big_axis[sgi];
    const unsigned int ax = T.axes[id];
    const unsigned int c = T.ntile[id], t0 = T.tile0[id], o = big_off[sgi];
    const unsigned int dst = T.sortbase[id] + (unsigned int)__popc(ax & ((1u << a) - 1u)) * c;
    const float4 cc = T.cen[id];
    const float3 u = axis_unit(a);
    for (unsigned int q = threadIdx.x; q < c; q += blockDim.x) {
      const unsigned int li = cval[o + q];
      sort_i[dst + q] = t0 + li;
      sort_r[dst + q] = tile_rlo(TL, T, t0 + li, cc, u);
    }
  }
}

}  // namespace sph
