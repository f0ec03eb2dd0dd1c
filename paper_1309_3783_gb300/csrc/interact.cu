// Density and force passes (Section II: two interaction stages), the ghost /
// h-update step between them, the FP64 conservation reductions and the
// per-field output gathers.
//
// Pair-interactions follow the sorted cell-pair interaction of Section II-C
// (Fig. 3) at warp granularity: particles are grouped into clusters of at most
// 32; a warp takes one cluster of cell A and walks the clusters of cell B in
// their sorted order along the axis joining the cell centres, stopping once the
// projected gap exceeds every support radius that could still bridge it, and
// culling clusters whose boxes are out of reach.  Each in-reach particle pair
// is found once and updates both sides (Section II-D: symmetric interactions).
#include "sph_engine.h"

#include <cfloat>
#include <mutex>

namespace sph {

constexpr float BAND_REL = 7.62939453125e-06f;  // 2^-17: guard band of the FP32 predicate

struct ItemGeom {
  float e;          // cell edge (units of L)
  float3 offB;      // centre of B minus centre of A (units of L), exact: e * db
  float offBp;      // projection of offB on the axis: e |db|
  float invL;
  float eb;         // length scale of the position rounding: the cell edge, or 1 (L) for
                    //   plain FP32 positions; the guard band is 2^-17 H (eb + H)
  float es;         // absolute rounding of plain FP32 positions added to the culling slack
  float L32;        // L in FP32
  float drift;      // largest displacement since the decomposition was built (units of L)
  double L, halfL;
  int periodic;
};

__device__ __forceinline__ ItemGeom item_geom(const Tree& T, const BoxDesc* box, int A, int ax) {
  ItemGeom g;
  const int d = T.level[A];
  const BoxDesc bd = box[T.box[A]];
  g.e = ldexpf(1.0f, -d);
  int dx, dy, dz;
  axis_vec(ax, dx, dy, dz);
  g.offB = make_float3(g.e * dx, g.e * dy, g.e * dz);
  const int n2 = dx * dx + dy * dy + dz * dz;
  g.offBp = g.e * (n2 == 1 ? 1.0f : (n2 == 2 ? 1.41421356237f : 1.73205080757f));
  g.invL = (float)bd.invL;
  g.eb = bd.global32 ? 1.0f : g.e;
  g.es = bd.global32 ? 9.5367431640625e-07f : 0.0f;   // 2^-20 L: the 2^-25 rounding of both positions
  g.L32 = (float)bd.L;
  g.drift = bd.drift_u;
  g.L = bd.L;
  g.halfL = 0.5 * bd.L;
  g.periodic = bd.periodic;
  return g;
}

// The FP64 data of a box that the exact decisions need, passed by value (an
// argument passed by reference to out-of-line code would live in local memory).
struct BoxExact {
  double L, halfL;
  int periodic;
};

__device__ __forceinline__ BoxExact box_exact(const ItemGeom& g) { return BoxExact{g.L, g.halfL, g.periodic}; }

// Tasks are handed out in chunks from a counter in device memory (zeroed before
// every launch): the cost of a task varies by orders of magnitude, so a static
// split leaves most SMs idle behind the longest ones.
// Consecutive tasks of a list mostly share their interaction (the clusters of one
// cell against the same partner cell), so a warp that takes several in a row finds
// the partners' data in its L1: the density pass, light per pair, gains from 8
// (33.5M: first pass 65.0 -> 62.7 ms); the force pass, heavy per pair, balances
// better with 2 (8 took it from 67.9 to 69.7 ms).
constexpr unsigned int TASK_CHUNK_DENSITY = 8;
constexpr unsigned int TASK_CHUNK_FORCE = 2;

// blocks per SM of the recording first density pass (5, with a few registers
// spilled for the record state, measured faster than 4 blocks without spills), of
// the plain first pass (see k_density) and of the later passes (5: with 5 % of the
// particles iterating, a later pass cost 26 % of a full pass unbounded at 3 blocks,
// 21 % at 5, 25 % at 7)
#ifndef REC_BLOCKS
#define REC_BLOCKS 5
#endif
#ifndef DENS_BLOCKS
#define DENS_BLOCKS 7
#endif
#ifndef PART_BLOCKS
#define PART_BLOCKS 5
#endif

// Exact decision r_ij < H (physical H) from the caller's FP64 positions.
__device__ __noinline__ bool exact_less(int gi, int gj, float Hphys, const unsigned int* __restrict__ perm,
                                        const double* __restrict__ x, double L, double halfL, int periodic) {
  const long long i = perm[gi], j = perm[gj];
  const double xi[3] = {x[3 * i], x[3 * i + 1], x[3 * i + 2]};
  const double xj[3] = {x[3 * j], x[3 * j + 1], x[3 * j + 2]};
  return canonical_less(canonical_r2(xi, xj, L, halfL, periodic), Hphys);
}

// FP32 test with guard band; inside the band the FP64 decision is taken.
__device__ __forceinline__ bool decide(float r2, float H2, float band, int gi, int gj, float Hphys,
                                       const unsigned int* perm, const double* x, const ItemGeom& g,
                                       unsigned int& rechecks) {
  const float dl = r2 - H2;
  if (dl < -band) return true;
  if (dl > band) return false;
  ++rechecks;
  return exact_less(gi, gj, Hphys, perm, x, g.L, g.halfL, g.periodic);
}

// =========================================================================== density
struct DensI {
  float3 p;
  float H, invH, H2, band, Hphys, m;
  int g;
  bool valid, act;
};

// The raw loads of one particle, issued ahead of their use (see the pair kernel).
struct DensRaw {
  float4 p, c;
  unsigned char a;
};

__device__ __forceinline__ DensRaw fetch_dens(bool valid, unsigned int gidx, const float4* pos4, const float4* cen4,
                                              const unsigned char* act) {
  DensRaw r;
  if (valid) {
    r.p = pos4[gidx];
    r.c = cen4[gidx];
    r.a = act ? act[gidx] : 1;      // no activity array: every particle iterates
  } else {
    r.p = make_float4(0.f, 0.f, 0.f, 0.f);
    r.c = r.p;
    r.a = 0;
  }
  return r;
}

__device__ __forceinline__ DensI make_dens(bool valid, unsigned int gidx, const DensRaw& raw, float3 shift,
                                           float invL, float e) {
  DensI r;
  r.valid = valid;
  if (valid) {
    const float4 p = raw.p;
    const float4 c = raw.c;
    // the cell offsets (c + shift) are exact dyadic values: add them first, round once
    r.p = make_float3(p.x + (c.x + shift.x), p.y + (c.y + shift.y), p.z + (c.z + shift.z));
    const float H = p.w * invL;
    r.H = H;
    r.invH = __fdividef(1.0f, H);   // 2 ulp: enters the kernel's argument only
    r.H2 = H * H;
    r.band = BAND_REL * H * (e + H);
    r.Hphys = p.w;
    r.m = c.w;
    r.g = (int)gidx;
    r.act = raw.a != 0;
  } else {
    r.p = make_float3(1e30f, 1e30f, 1e30f);
    r.H = 0.0f;
    r.invH = 0.0f;
    r.H2 = -1.0f;
    r.band = 0.0f;
    r.Hphys = 0.0f;
    r.m = 0.0f;
    r.g = -1;
    r.act = false;
  }
  return r;
}

__device__ __forceinline__ DensI load_dens(bool valid, unsigned int gidx, float3 shift, const float4* pos4,
                                           const float4* cen4, const unsigned char* act, float invL, float e) {
  return make_dens(valid, gidx, fetch_dens(valid, gidx, pos4, cen4, act), shift, invL, e);
}

// Per warp: the staged partners (p, a, g, act) and the warp's own cluster (ip).
struct DensShared {
  float4 p[32];     // partner position, H^2 (units of L; H^2 = -1 marks an empty slot)
  float4 a[32];     // partner 1/H, band, m, H (physical)
  int g[32];
  unsigned char act[32];
  float4 ip[32];    // own cluster: position, m
  // pair records (first pass): the current task's first batch, batch count and
  // record slot, and 0 once one of its batches was lost (lane 0 keeps them)
  unsigned int rc_first, rc_nb, rc_slot, rc_ok;
};

// A warp's next batch (first pass, the same in every lane); a multiple of
// REC_CHUNK means that its chunk is used up (0: no chunk yet).
struct RecW {
  unsigned int pos = 0;
};

__device__ __forceinline__ void dens_put(DensShared& S, int lane, const DensI& j) {
  S.p[lane] = make_float4(j.p.x, j.p.y, j.p.z, j.H2);
  S.a[lane] = make_float4(j.invH, j.band, j.m, j.Hphys);
  S.g[lane] = j.g;
  S.act[lane] = j.act ? 1 : 0;
}

__device__ __forceinline__ void dens_stage_own(DensShared& S, int lane, const DensI& i) {
  S.ip[lane] = make_float4(i.p.x, i.p.y, i.p.z, i.m);
}

struct Counters {
  unsigned int cand = 0, pairs = 0, sides = 0, rechecks = 0;
};

// A later pass of the h iteration gathers (the symmetric tasks stand aside) when
// its task builder chose to and its tasks fitted the buffer.
__device__ __forceinline__ bool gather_on(const int* gflag, const unsigned int* g_n, unsigned int cap_g) {
  return gflag[0] != 0 && *g_n <= cap_g;
}

__device__ __forceinline__ void flush_dens(int gidx, float4 acc, unsigned int cnt, float4* dacc, unsigned int* dcnt) {
  if (gidx < 0 || cnt == 0) return;
  atomicAdd(&dacc[gidx], acc);
  atomicAdd(&dcnt[gidx], cnt);
}

template <bool COUNT>
__device__ __forceinline__ void commit_counters(const Counters& C, unsigned long long* pc, int which) {
  if (!COUNT) return;
  unsigned long long c = C.cand, p = C.pairs, s = C.sides, r = C.rechecks;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    c += __shfl_xor_sync(0xffffffffu, c, o);
    p += __shfl_xor_sync(0xffffffffu, p, o);
    s += __shfl_xor_sync(0xffffffffu, s, o);
    r += __shfl_xor_sync(0xffffffffu, r, o);
  }
  if ((threadIdx.x & 31) == 0) {
    // pc: [0..2] density cell-pair kernel (pairs, sides, candidates), [3..5] density
    // self kernel, [6..7] force cell-pair kernel (pairs, candidates), [8..9] force
    // self kernel, [10] FP64 re-decisions
    const int base = which == 0 ? 0 : which == 1 ? 3 : which == 2 ? 6 : 8;
    atomicAdd(&pc[base], p);
    if (which < 2) atomicAdd(&pc[base + 1], s);
    atomicAdd(&pc[base + (which < 2 ? 2 : 1)], c);
    atomicAdd(&pc[10], r);
  }
}


// the lanes above this one
__device__ __forceinline__ unsigned int upper_mask(int lane) {
  return lane == 31 ? 0u : (0xffffffffu << (lane + 1));
}

// ------------------------------------------------------------- pair records
// Called by the whole warp.  A task starts with no batch; its batches go to the
// warp's current chunk, and to a new chunk (linked from the old one) when that is
// full.  A batch that finds the pool full is lost, and with it the task's record.
__device__ __forceinline__ void rec_task_begin(DensShared& S, unsigned int slot) {
  if ((threadIdx.x & 31) == 0) {
    S.rc_nb = 0;
    S.rc_ok = 1;
    S.rc_slot = slot;
  }
}

__device__ __forceinline__ void rec_batch(const PairRec& R, RecW& W, DensShared& S, unsigned int jvalid,
                                          unsigned int m) {
  const int lane = threadIdx.x & 31;
  __syncwarp();
  if (!S.rc_ok) return;
  if (W.pos % REC_CHUNK == 0u) {
    unsigned int c = 0;
    if (lane == 0) c = atomicAdd(R.ctr, 1u);
    c = __shfl_sync(0xffffffffu, c, 0);
    if (c >= R.cap) {
      if (lane == 0) S.rc_ok = 0;
      W.pos = 0;
      return;
    }
    if (lane == 0 && W.pos != 0) R.next[W.pos / REC_CHUNK - 1u] = c;
    W.pos = c * REC_CHUNK;
  }
  // streaming stores: the records are read once, by the force pass, and should
  // not push the particle data the passes share out of L2
  unsigned int* B = R.pool + 64ull * W.pos;
  __stcs(B + lane, (jvalid >> lane) & 1u ? (unsigned int)S.g[lane] : REC_NONE);
  __stcs(B + 32 + lane, m);
  if (lane == 0) {
    if (S.rc_nb == 0) S.rc_first = W.pos;
    S.rc_nb += 1;
  }
  W.pos += 1;
}

__device__ __forceinline__ void rec_task_end(uint2* slots, const DensShared& S) {
  __syncwarp();
  if ((threadIdx.x & 31) == 0 && S.rc_ok) slots[S.rc_slot] = make_uint2(S.rc_nb ? S.rc_first : 0u, S.rc_nb);
}

// =========================================================================== force
struct ForceI {
  float3 p;
  float H, invH, H2, band, Hphys, m;
  float3 v;
  float rho, F, c, K4;
  int g;
  bool valid;
};

__device__ __forceinline__ ForceI load_force(bool valid, unsigned int gidx, float3 shift, const float4* pos4,
                                             const float4* cen4, const float4* vel4, const float4* ghost4,
                                             float invL, float L, float e) {
  ForceI r;
  r.valid = valid;
  if (valid) {
    const float4 p = pos4[gidx];
    const float4 c = cen4[gidx];
    const float4 vv = vel4[gidx];
    const float4 gh = ghost4[gidx];
    // the cell offsets (c + shift) are exact dyadic values: add them first, round once
    r.p = make_float3(p.x + (c.x + shift.x), p.y + (c.y + shift.y), p.z + (c.z + shift.z));
    const float H = p.w * invL;
    r.H = H;
    r.invH = gh.w * L;                // 1 / H in units of L
    r.H2 = H * H;
    r.band = BAND_REL * H * (e + H);
    r.Hphys = p.w;
    r.m = c.w;
    r.v = make_float3(vv.x, vv.y, vv.z);
    r.rho = gh.x;
    r.F = gh.y;
    r.c = gh.z;
    const float ih = gh.w;            // 1 / H (physical), from the ghost pass
    r.K4 = SPH_KNORM * (ih * ih) * (ih * ih);
    r.g = (int)gidx;
  } else {
    r.p = make_float3(1e30f, 1e30f, 1e30f);
    r.H = 0.f;
    r.invH = 0.f;
    r.H2 = -1.f;
    r.band = 0.f;
    r.Hphys = 0.f;
    r.m = 0.f;
    r.v = make_float3(0.f, 0.f, 0.f);
    r.rho = 1.f;
    r.F = 0.f;
    r.c = 0.f;
    r.K4 = 0.f;
    r.g = -1;
  }
  return r;
}

// Per warp: the staged partners (p, a, v, f, g) and the warp's own cluster
// (ip, iv, if_).  The pair list holds 768 of a batch's up to 1024 pairs, so that
// 8 blocks of 4 warps fit an SM's shared memory (the register cap's occupancy; with
// a full list shared memory held the kernel at 7 blocks, 3.5 % slower on the 33.5M
// box); a batch with more pairs runs as two halves of the own lanes.
constexpr int PLIST_CAP = 768;
struct ForceShared {
  float4 p[32];    // partner position, H^2
  float4 a[32];    // partner 1/H, band, m, H (physical)
  float4 v[32];    // partner velocity, rho
  float4 f[32];    // partner f P / rho^2, c, K/H^4, -
  float4 jacc[32]; // partner sums of the batch: acceleration (3), du/dt (their largest
                   //   signal velocity in f[].w)
  int g[32];
  float4 ip[32];   // own cluster: position, m
  float4 iv[32];   // own cluster: velocity, rho
  float4 if_[32];  // own cluster: 1/H, f P / rho^2, c, K/H^4
  float4 ih[32];   // own cluster: H^2 (-1: no particle), band, H (physical), index (bits)
  float4 iacc[32]; // own cluster sums over the task
  float ivs[32];
  unsigned short plist[PLIST_CAP]; // the batch's pairs: own lane | slot << 5
};

__device__ __forceinline__ void force_put(ForceShared& S, int lane, const ForceI& j) {
  S.p[lane] = make_float4(j.p.x, j.p.y, j.p.z, j.H2);
  S.a[lane] = make_float4(j.invH, j.band, j.m, j.Hphys);
  S.v[lane] = make_float4(j.v.x, j.v.y, j.v.z, j.rho);
  S.f[lane] = make_float4(j.F, j.c, j.K4, 0.f);   // w: the partner's largest v_sig of the batch
  S.jacc[lane] = make_float4(0.f, 0.f, 0.f, 0.f);
  S.g[lane] = j.g;
}

__device__ __forceinline__ void force_stage_own(ForceShared& S, int lane, const ForceI& i) {
  S.ip[lane] = make_float4(i.p.x, i.p.y, i.p.z, i.m);
  S.iv[lane] = make_float4(i.v.x, i.v.y, i.v.z, i.rho);
  S.if_[lane] = make_float4(i.invH, i.F, i.c, i.K4);
  S.ih[lane] = make_float4(i.valid ? i.H2 : -1.0f, i.band, i.Hphys, __int_as_float(i.g));
  S.iacc[lane] = make_float4(0.f, 0.f, 0.f, 0.f);
  S.ivs[lane] = 0.f;
}

__device__ __forceinline__ void flush_force(int gidx, float4 acc, float vs, float4* facc, float* fvsig) {
  if (gidx < 0 || !(vs > 0.0f)) return;   // vsig > 0 for every pair that contributed
  atomicAdd(&facc[gidx], acc);
  atomic_max_pos(&fvsig[gidx], vs);
}

// ------------------------------------------------------------- two-phase tiles
// Up to 32 partners sit in shared memory: particles of one or several partner
// clusters that passed a test against the box of the warp's cluster.  Phase 1:
// every lane tests its particle i against the staged partners (broadcast
// reads) and keeps two bitmasks, r < H_i and r < H_j, decided exactly.  Phase 2
// runs two sweeps without atomics: in the row sweep every lane walks its own
// bits and accumulates its own side; the r < H_j mask is then transposed with
// ballots so that in the column sweep every staged partner walks the lanes it
// interacts with and accumulates its side in registers, flushed once to global
// memory.  Each in-reach pair is still found once and updates both sides.
// Inside one cluster (own-only batches) every lane walks its full row for its
// own side, which keeps the lanes balanced: each pair's two sides are then
// computed by the two lanes concerned.  Invalid lanes sit at 1e30 with
// H^2 = -1, so they never pass a test.

// Phase 1: exact bitmasks of r < H_i (mI) and r < H_j (mJ) over the first n
// staged partners (n a multiple of 4; slots past the batch hold empty entries).
// The FP32 test decides outside a guard band around H^2; bandJ bounds every
// partner's band; the few uncertain bits are decided in FP64 afterwards.
template <class SH>
__device__ __forceinline__ void pair_masks(const float3 ip, float iH2, float iband, int ig, float iHphys,
                                           const SH& S, float bandJ, unsigned int allow, int n,
                                           const unsigned int* perm, const double* x, const BoxExact g,
                                           unsigned int& mI, unsigned int& mJ, unsigned int& rc) {
  // Per slot, r^2 against H^2 - band (sure inside) and H^2 + band (sure outside),
  // for both radii: each test is the sign of one difference, shifted into its mask
  // (slots taken from the last, so that slot s lands in bit s).  u: slots where
  // either decision is not sure; both are then taken again in FP64 (the exact
  // decision equals the FP32 one where that was sure).
  const float iLo = iH2 - iband, iHi = iH2 + iband;
  unsigned int sure = 0;   // slots where both decisions are sure
  mI = 0;
  mJ = 0;
  for (int s0 = n - 4; s0 >= 0; s0 -= 4) {
#pragma unroll
    for (int k = 3; k >= 0; --k) {
      const int s = s0 + k;
      const float4 J = S.p[s];
      const float dx = ip.x - J.x, dy = ip.y - J.y, dz = ip.z - J.z;
      const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
      const unsigned int ai = __float_as_uint(r2 - iLo), bi = __float_as_uint(iHi - r2);   // sign: in / out
      const unsigned int aj = __float_as_uint(r2 - (J.w - bandJ)), bj = __float_as_uint((J.w + bandJ) - r2);
      mI = __funnelshift_l(ai, mI, 1);
      mJ = __funnelshift_l(aj, mJ, 1);
      sure = __funnelshift_l((ai | bi) & (aj | bj), sure, 1);
    }
  }
  unsigned int u = ~sure & allow;
  while (u) {
    const int s = __ffs(u) - 1;
    u &= u - 1;
    rc += 2;
    const unsigned int bit = 1u << s;
    mI = exact_less(ig, S.g[s], iHphys, perm, x, g.L, g.halfL, g.periodic) ? (mI | bit) : (mI & ~bit);
    mJ = exact_less(ig, S.g[s], S.a[s].w, perm, x, g.L, g.halfL, g.periodic) ? (mJ | bit) : (mJ & ~bit);
  }
  mI &= allow;
  mJ &= allow;
}

// lane s receives the lanes whose mask has bit s: the 32 x 32 bit matrix (row =
// lane) transposed by recursive exchange of its off-diagonal blocks, 16 x 16
// down to 1 x 1, one shuffle per level.
__device__ __forceinline__ unsigned int transpose_bits(unsigned int m) {
  const int lane = threadIdx.x & 31;
  unsigned int x = m;
#pragma unroll
  for (int j = 16; j > 0; j >>= 1) {
    const unsigned int mk = j == 16 ? 0x0000FFFFu : j == 8 ? 0x00FF00FFu : j == 4 ? 0x0F0F0F0Fu
                          : j == 2 ? 0x33333333u : 0x55555555u;
    const unsigned int y = __shfl_xor_sync(0xffffffffu, x, j);
    x = (lane & j) ? ((x & ~mk) | ((y & ~mk) >> j)) : ((x & mk) | ((y & mk) << j));
  }
  return x;
}

// The four density sums of a particle (sum m w, sum m q w', sum w, sum q w').
// KAHAN: compensated (Neumaier) summation, for high neighbour counts: each sum
// carries the rounding errors of its additions in c, and the total is s + c, so
// its error no longer grows with the number of terms.
template <bool KAHAN>
struct DensAcc {
  float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
  float4 c = make_float4(0.f, 0.f, 0.f, 0.f);
  __device__ __forceinline__ static void kadd(float& sum, float& comp, float x) {
    const float t = sum + x;
    comp += fabsf(sum) >= fabsf(x) ? (sum - t) + x : (x - t) + sum;
    sum = t;
  }
  __device__ __forceinline__ void add(float m, float w, float gg) {
    if (KAHAN) {
      kadd(s.x, c.x, m * w);
      kadd(s.y, c.y, m * gg);
      kadd(s.z, c.z, w);
      kadd(s.w, c.w, gg);
    } else {
      s.x = fmaf(m, w, s.x);
      s.y = fmaf(m, gg, s.y);
      s.z += w;
      s.w += gg;
    }
  }
  __device__ __forceinline__ float4 total() const {
    return KAHAN ? make_float4(s.x + c.x, s.y + c.y, s.z + c.z, s.w + c.w) : s;
  }
};

// r from r^2 by the fast reciprocal square root (its rounding enters the kernel's
// argument only; the neighbour decision is taken on r^2)
__device__ __forceinline__ float pair_r(float r2) { return r2 > 0.0f ? r2 * rsqrtf(r2) : 0.0f; }

// One density contribution: w and q w'(q) at q = r / H, weighted by m.
template <bool KAHAN>
__device__ __forceinline__ void dens_add(float r, float invH, float m, DensAcc<KAHAN>& acc, unsigned int& cnt) {
  float w, dw;
  const float q = r * invH;
  spline_w_dw(q, w, dw);
  const float gg = q * dw;                 // q w'(q) = r dW/dr in units of W
  acc.add(m, w, gg);
  cnt++;
}

// Density batch: own side for r < H_i (active i), partner side for r < H_j
// (active j) unless own_only.  cmask selects the bits the counters count (the
// upper triangle inside one cluster, where every pair appears in both rows).
template <bool COUNT, bool KAHAN>
__device__ __forceinline__ void dens_tile(const DensI& I, DensShared& S, unsigned int allow, unsigned int jvalid,
                                          unsigned int jact, float bandJ, int n, bool own_only, unsigned int cmask,
                                          DensAcc<KAHAN>& acc, unsigned int& cnt, const unsigned int* perm,
                                          const double* x, const ItemGeom& g, float4* dacc, unsigned int* dcnt,
                                          Counters& C, bool rec, const PairRec& R, RecW& W) {
  const int lane = threadIdx.x & 31;
  unsigned int mI, mJ, rc = 0;
  pair_masks(I.p, I.H2, I.band, I.g, I.Hphys, S, bandJ, allow, n, perm, x, box_exact(g), mI, mJ, rc);
  // the pairs for the force pass: each unordered pair once (inside one cluster,
  // the partners above the lane)
  if (rec) rec_batch(R, W, S, jvalid, (mI | mJ) & (own_only ? upper_mask(lane) : 0xffffffffu));
  const unsigned int ui = I.act ? mI : 0u, uj = own_only ? 0u : (mJ & jact);
  if (COUNT) {
    C.cand += I.valid ? __popc(allow & jvalid & cmask) : 0u;
    C.rechecks += rc;
    C.pairs += __popc((ui | (mJ & jact)) & cmask);
    C.sides += __popc(ui) + __popc(uj);
  }
  // row sweep: own side
  for (unsigned int m = ui; m; m &= m - 1) {
    const int sj = __ffs(m) - 1;
    const float4 J = S.p[sj];
    const float dx = I.p.x - J.x, dy = I.p.y - J.y, dz = I.p.z - J.z;
    dens_add(pair_r(fmaf(dz, dz, fmaf(dy, dy, dx * dx))), I.invH, S.a[sj].z, acc, cnt);
  }
  if (own_only) return;
  // column sweep: partner side, staged partner = lane
  unsigned int col = transpose_bits(uj);
  if (col) {
    const float4 J = S.p[lane];
    const float jinvH = S.a[lane].x;
    DensAcc<KAHAN> pacc;
    unsigned int pcnt = 0;
    for (; col; col &= col - 1) {
      const int li = __ffs(col) - 1;
      const float4 P = S.ip[li];
      const float dx = P.x - J.x, dy = P.y - J.y, dz = P.z - J.z;
      dens_add(pair_r(fmaf(dz, dz, fmaf(dy, dy, dx * dx))), jinvH, P.w, pacc, pcnt);
    }
    flush_dens(S.g[lane], pacc.total(), pcnt, dacc, dcnt);
  }
}

// What one side of a force pair needs of a particle: position, velocity, rho,
// f P / rho^2, sound speed, K/H^4, 1/H and mass.
struct ForceSide {
  float3 p, v;
  float rho, F, c, K4, invH, m;
};

// Both sides of one force pair, a (own particle) and b (partner), d = x_a - x_b:
// a gains ca, b gains cb (the antisymmetric acceleration terms and each side's
// du/dt), both see vsig.  No contribution when r = 0.  A side's kernel gradient
// is taken inside its support (q < 1) and is zero outside; at q = 1 it is zero
// too, so the FP32 test agrees with the exact one to within the gradient's size
// there, about 6 (1 - q)^2 for q within rounding of 1.
__device__ __forceinline__ void force_pair_terms(const ForceSide& a, const ForceSide& b,
                                                 float alpha, float4& ca, float4& cb, float& vsig) {
  const float dx = a.p.x - b.p.x, dy = a.p.y - b.p.y, dz = a.p.z - b.p.z;
  const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
  ca = make_float4(0.f, 0.f, 0.f, 0.f);
  cb = ca;
  vsig = 0.0f;
  if (!(r2 > 0.0f)) return;
  const float rinv = rsqrtf(r2);
  const float r = r2 * rinv;
  float w, dwa, dwb;
  const float qa = r * a.invH, qb = r * b.invH;
  spline_w_dw(qa, w, dwa);
  spline_w_dw(qb, w, dwb);
  dwa = qa < 1.0f ? dwa : 0.0f;
  dwb = qb < 1.0f ? dwb : 0.0f;
  const float Wa = a.K4 * dwa, Wb = b.K4 * dwb;
  const float vdx = fmaf(a.v.x - b.v.x, dx, fmaf(a.v.y - b.v.y, dy, (a.v.z - b.v.z) * dz));
  const float wv = vdx * rinv;
  const float mu = fminf(wv, 0.0f);
  vsig = a.c + b.c - 3.0f * mu;
  const float Pi = __fdividef(-alpha * vsig * mu, a.rho + b.rho);
  const float Wbar = 0.5f * (Wa + Wb);
  const float coef = fmaf(a.F, Wa, fmaf(b.F, Wb, Pi * Wbar)) * rinv;
  const float hv = 0.5f * Pi * Wbar;
  const float ka = -b.m * coef, kb = a.m * coef;
  ca = make_float4(ka * dx, ka * dy, ka * dz, b.m * fmaf(a.F, Wa, hv) * wv);
  cb = make_float4(kb * dx, kb * dy, kb * dz, a.m * fmaf(b.F, Wb, hv) * wv);
}

// Sums over runs of adjacent lanes with the same key; true on the first lane of
// each run, which then holds the run's total (sum of v, max of m).
__device__ __forceinline__ bool run_sum_max(int key, float4& v, float& m) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const int k2 = __shfl_down_sync(0xffffffffu, key, off);
    const float x = __shfl_down_sync(0xffffffffu, v.x, off), y = __shfl_down_sync(0xffffffffu, v.y, off);
    const float z = __shfl_down_sync(0xffffffffu, v.z, off), w = __shfl_down_sync(0xffffffffu, v.w, off);
    const float m2 = __shfl_down_sync(0xffffffffu, m, off);
    if (lane + off < 32 && k2 == key) {
      v.x += x;
      v.y += y;
      v.z += z;
      v.w += w;
      m = fmaxf(m, m2);
    }
  }
  const int prev = __shfl_up_sync(0xffffffffu, key, 1);   // every lane takes part in the shuffle
  return lane == 0 || prev != key;
}

__device__ __forceinline__ ForceSide side_of(const ForceI& I) {
  ForceSide s;
  s.p = I.p;
  s.v = I.v;
  s.rho = I.rho;
  s.F = I.F;
  s.c = I.c;
  s.K4 = I.K4;
  s.invH = I.invH;
  s.m = I.m;
  return s;
}

__device__ __forceinline__ ForceSide staged_side(const ForceShared& S, int k) {
  const float4 P = S.p[k], A = S.a[k], V = S.v[k], F = S.f[k];
  ForceSide s;
  s.p = make_float3(P.x, P.y, P.z);
  s.v = make_float3(V.x, V.y, V.z);
  s.rho = V.w;
  s.F = F.x;
  s.c = F.y;
  s.K4 = F.z;
  s.invH = A.x;
  s.m = A.z;
  return s;
}

__device__ __forceinline__ ForceSide own_side(const ForceShared& S, int k) {
  const float4 P = S.ip[k], V = S.iv[k], F = S.if_[k];
  ForceSide s;
  s.p = make_float3(P.x, P.y, P.z);
  s.v = make_float3(V.x, V.y, V.z);
  s.rho = V.w;
  s.invH = F.x;
  s.F = F.y;
  s.c = F.z;
  s.K4 = F.w;
  s.m = P.w;
  return s;
}

// The pairs of one batch (mask m of the lane's own particle over the staged
// slots), each evaluated once for both sides.  The pairs go into a list in shared
// memory (own lane major), which the warp then takes 32 at a time: one pair per
// lane, so that all lanes work however unevenly the pairs fall on the rows.  The
// own side is summed by a segmented warp reduction (a particle's pairs are
// adjacent in the list) into its task sums; the partner side goes to the
// partner's batch sums (or, inside one cluster, to that particle's task sums).
template <bool COUNT>
__device__ __forceinline__ void force_rounds_list(ForceShared& S, unsigned int m, bool own_only, float alpha,
                                                  unsigned int* fcnt, unsigned int cnt, unsigned int incl,
                                                  unsigned int total);

// A batch with more pairs than the list holds (rare: dense clusters): two halves
// of the own lanes, at most 16 x 32 pairs each, out of line so that the common
// path keeps its registers.
template <bool COUNT>
__device__ __noinline__ void force_rounds_halves(ForceShared& S, unsigned int m, bool own_only, float alpha,
                                                 unsigned int* fcnt) {
  const int lane = threadIdx.x & 31;
  for (int half = 0; half < 2; ++half) {
    const unsigned int mh = (lane >> 4) == half ? m : 0u;
    const unsigned int ch = __popc(mh);
    unsigned int ih = ch;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned int y = __shfl_up_sync(0xffffffffu, ih, o);
      if (lane >= o) ih += y;
    }
    force_rounds_list<COUNT>(S, mh, own_only, alpha, fcnt, ch, ih, __shfl_sync(0xffffffffu, ih, 31));
  }
}

template <bool COUNT>
__device__ __forceinline__ void force_rounds(ForceShared& S, unsigned int m, bool own_only, float alpha,
                                             unsigned int* fcnt) {
  const int lane = threadIdx.x & 31;
  // list the pairs, own lane major (in two halves of the own lanes when they do
  // not fit the list: at most 16 x 32 pairs each)
  const unsigned int cnt = __popc(m);
  unsigned int incl = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  const unsigned int total = __shfl_sync(0xffffffffu, incl, 31);
  if (total <= (unsigned int)PLIST_CAP) force_rounds_list<COUNT>(S, m, own_only, alpha, fcnt, cnt, incl, total);
  else force_rounds_halves<COUNT>(S, m, own_only, alpha, fcnt);
}

// The rounds over one list: cnt pairs of the lane (mask m), incl their inclusive
// prefix over the lanes, total all of them (<= PLIST_CAP).
template <bool COUNT>
__device__ __forceinline__ void force_rounds_list(ForceShared& S, unsigned int m, bool own_only, float alpha,
                                                  unsigned int* fcnt, unsigned int cnt, unsigned int incl,
                                                  unsigned int total) {
  const int lane = threadIdx.x & 31;
  __syncwarp();
  unsigned int k = incl - cnt;
  for (unsigned int mm = m; mm; mm &= mm - 1) {
    const unsigned int sj = __ffs(mm) - 1;
    S.plist[k++] = (unsigned short)(lane | (sj << 5));
  }
  __syncwarp();
  const unsigned int lt = (1u << lane) - 1u;
  for (unsigned int r0 = 0; r0 < total; r0 += 32) {
    const unsigned int e = r0 + lane;
    int li = 32 + lane;     // a key no other lane has
    float4 ci = make_float4(0.f, 0.f, 0.f, 0.f), cj = ci;
    float vs = 0.0f;
    int sj = 64 + lane;     // likewise
    if (e < total) {
      const unsigned int w = S.plist[e];
      li = (int)(w & 31u);
      sj = (int)((w >> 5) & 31u);
      force_pair_terms(own_side(S, li), staged_side(S, sj), alpha, ci, cj, vs);
      if (COUNT) {
        // force partners of both particles (the pair set, checked per particle)
        atomicAdd(&fcnt[__float_as_int(S.ih[li].w)], 1u);
        atomicAdd(&fcnt[S.g[sj]], 1u);
      }
    }
    // Shared-memory float atomics are slow, the more so where lanes collide, so
    // the sums are written plainly in steps that touch each particle once.  Own
    // side: one head lane per row of the round holds the row's total.
    float vmax = vs;
    if (run_sum_max(li, ci, vmax) && li < 32) {
      float4 t = S.iacc[li];
      t.x += ci.x; t.y += ci.y; t.z += ci.z; t.w += ci.w;
      S.iacc[li] = t;
      atomicMax(reinterpret_cast<unsigned int*>(&S.ivs[li]), __float_as_uint(vmax));
    }
    __syncwarp();
    // partner side: the lanes of one partner take turns by their rank among them
    const unsigned int peers = __match_any_sync(0xffffffffu, sj);
    const unsigned int rank = __popc(peers & lt);
    const unsigned int nturn = __reduce_max_sync(0xffffffffu, e < total ? rank : 0u);
    float4* dst = own_only ? S.iacc : S.jacc;
    for (unsigned int r = 0; r <= nturn; ++r) {
      if (e < total && rank == r) {
        float4 t = dst[sj];
        t.x += cj.x; t.y += cj.y; t.z += cj.z; t.w += cj.w;
        dst[sj] = t;
      }
      __syncwarp();
    }
    if (e < total) atomicMax(reinterpret_cast<unsigned int*>(own_only ? &S.ivs[sj] : &S.f[sj].w), __float_as_uint(vs));
    __syncwarp();
  }
}

// Force batch: every pair with r < max(H_i, H_j) among the staged partners,
// decided exactly (phase 1), then evaluated for both sides.
template <bool COUNT>
__device__ __forceinline__ void force_tile(ForceShared& S, unsigned int allow, unsigned int jvalid,
                                           float bandJ, int n, bool own_only, unsigned int cmask,
                                           const unsigned int* perm, const double* x, const BoxExact g,
                                           float alpha, unsigned int* fcnt, Counters* C) {
  // the lane's own particle, read back from the staged cluster
  const float4 ip = S.ip[threadIdx.x & 31], ih = S.ih[threadIdx.x & 31];
  const bool ivalid = ih.x >= 0.0f;
  unsigned int mI, mJ, rc = 0;
  pair_masks(make_float3(ip.x, ip.y, ip.z), ih.x, ih.y, __float_as_int(ih.w), ih.z, S, bandJ, allow, n, perm, x, g,
             mI, mJ, rc);
  const unsigned int m = mI | mJ;
  if (COUNT) {
    C->cand += ivalid ? __popc(allow & jvalid & cmask) : 0u;
    C->rechecks += rc;
    C->pairs += __popc(m & cmask);
  }
  force_rounds<COUNT>(S, m, own_only, alpha, fcnt);
}

// One batch of q <= 32 staged partners (slots 0..q-1) against the warp's
// cluster: empty the slots past the batch and run both phases over the first
// q rounded up to 4.  own_only: the partners are the warp's own cluster (each
// lane excludes itself and updates its own side only).
template <bool COUNT, bool PART, bool KAHAN, bool REC>
__device__ __forceinline__ void dens_batch(const DensI& I, DensShared& S, unsigned int q, bool own_only,
                                           DensAcc<KAHAN>& acc, unsigned int& cnt, const unsigned int* perm,
                                           const double* x, const ItemGeom& g, float4* dacc, unsigned int* dcnt,
                                           Counters& C, const PairRec& R, RecW& W) {
  const int lane = threadIdx.x & 31;
  const bool v = (unsigned int)lane < q;
  __syncwarp();
  if (!v) S.p[lane] = make_float4(1e30f, 1e30f, 1e30f, -1.0f);
  const unsigned int jvalid = __ballot_sync(0xffffffffu, v);
  const unsigned int jact = PART ? __ballot_sync(0xffffffffu, v && S.act[lane]) : jvalid;
  const float bandJ = warp_max(v ? S.a[lane].y : 0.0f);
  __syncwarp();
  const unsigned int allow = own_only ? jvalid & ~(1u << lane) : jvalid;
  dens_tile<COUNT, KAHAN>(I, S, allow, jvalid, jact, bandJ, (int)((q + 3u) & ~3u), own_only,
                   own_only ? upper_mask(lane) : 0xffffffffu, acc, cnt, perm, x, g, dacc, dcnt, C, REC && !PART, R, W);
  __syncwarp();
}

// Not inlined: the pair and self tasks share one copy of the batch code, which
// keeps the force kernel's instructions within the instruction cache (inlined
// twice, instruction fetch was the largest stall of the kernel).  Everything is
// passed by value or by pointer, so that a call stores nothing to local memory.
template <bool COUNT>
__device__ __noinline__ void force_batch(ForceShared& S, unsigned int q, bool own_only,
                                            const unsigned int* perm, const double* x, const BoxExact g,
                                            float alpha, float4* facc, float* fvsig, unsigned int* fcnt,
                                            Counters* C) {
  const int lane = threadIdx.x & 31;
  const bool v = (unsigned int)lane < q;
  __syncwarp();
  if (!v) S.p[lane] = make_float4(1e30f, 1e30f, 1e30f, -1.0f);
  const unsigned int jvalid = __ballot_sync(0xffffffffu, v);
  const float bandJ = warp_max(v ? S.a[lane].y : 0.0f);
  __syncwarp();
  // inside one cluster each unordered pair once (partners above the lane)
  const unsigned int allow = own_only ? jvalid & upper_mask(lane) : jvalid;
  force_tile<COUNT>(S, allow, jvalid, bandJ, (int)((q + 3u) & ~3u), own_only, 0xffffffffu, perm, x, g, alpha,
                    fcnt, C);
  __syncwarp();
  if (v && !own_only) flush_force(S.g[lane], S.jacc[lane], S.f[lane].w, facc, fvsig);
  __syncwarp();
}

// One recorded batch B of the first density pass: the staged partners are read
// back by index (own_only: the warp's own cluster, already staged), the pairs come
// from the recorded masks, and phase 2 runs as in force_batch.
template <bool COUNT>
__device__ __noinline__ void force_replay_batch(ForceShared& S, const unsigned int* __restrict__ B, bool own_only,
                                                float3 sh, float invL, float L32, float eb,
                                                const float4* __restrict__ pos4, const float4* __restrict__ cen4,
                                                const float4* __restrict__ vel4, const float4* __restrict__ ghost4,
                                                float alpha, float4* facc, float* fvsig, unsigned int* fcnt,
                                                Counters* C) {
  const int lane = threadIdx.x & 31;
  const unsigned int gj = __ldcs(B + lane);     // read once: evict first
  const unsigned int m = __ldcs(B + 32 + lane);
  const bool v = gj != REC_NONE;
  __syncwarp();
  if (!own_only) force_put(S, lane, load_force(v, gj, sh, pos4, cen4, vel4, ghost4, invL, L32, eb));
  __syncwarp();
  if (COUNT) {
    const unsigned int jvalid = __ballot_sync(0xffffffffu, v);
    C->cand += S.ih[lane].x >= 0.0f ? __popc(jvalid & (own_only ? upper_mask(lane) : 0xffffffffu)) : 0u;
    C->pairs += __popc(m);
  }
  force_rounds<COUNT>(S, m, own_only, alpha, fcnt);
  __syncwarp();
  if (v && !own_only) flush_force(S.g[lane], S.jacc[lane], S.f[lane].w, facc, fvsig);
  __syncwarp();
}

// ------------------------------------------------------------- cluster geometry
__device__ __forceinline__ float3 axis_unit_f(int a) {
  int dx, dy, dz;
  axis_vec(a, dx, dy, dz);
  const int n2 = dx * dx + dy * dy + dz * dz;
  const float s = n2 == 1 ? 1.0f : (n2 == 2 ? 0.70710678118654752f : 0.57735026918962576f);
  return make_float3(dx * s, dy * s, dz * s);
}

struct Box3 {
  float3 lo, hi;
};

// box of cluster t in the frame whose origin sits at -off from the leaf frame:
// box + (leaf centre + off), the offset being exact (dyadic)
__device__ __forceinline__ Box3 tile_box3(const Tiles& TL, const Tree& T, unsigned int t, float3 off) {
  const float4 lc = TL.cen[t];
  const float4 lo = TL.lo[t], hi = TL.hi[t];
  const float ox = lc.x + off.x, oy = lc.y + off.y, oz = lc.z + off.z;
  Box3 b;
  b.lo = make_float3(lo.x + ox, lo.y + oy, lo.z + oz);
  b.hi = make_float3(hi.x + ox, hi.y + oy, hi.z + oz);
  return b;
}

// Distance between two boxes within reach, compared squared (FP32; the
// caller's slack, at least 1e-6 of the reach, covers the rounding of both forms).
__device__ __forceinline__ bool box_near(const Box3& a, const Box3& b, float reach) {
  const float gx = fmaxf(0.0f, fmaxf(b.lo.x - a.hi.x, a.lo.x - b.hi.x));
  const float gy = fmaxf(0.0f, fmaxf(b.lo.y - a.hi.y, a.lo.y - b.hi.y));
  const float gz = fmaxf(0.0f, fmaxf(b.lo.z - a.hi.z, a.lo.z - b.hi.z));
  return fmaf(gx, gx, fmaf(gy, gy, gz * gz)) <= reach * reach;
}

// distance from a point to a box within reach (as box_near)
__device__ __forceinline__ bool near_box(const float3 p, const Box3& b, float reach) {
  const float gx = fmaxf(0.0f, fmaxf(b.lo.x - p.x, p.x - b.hi.x));
  const float gy = fmaxf(0.0f, fmaxf(b.lo.y - p.y, p.y - b.hi.y));
  const float gz = fmaxf(0.0f, fmaxf(b.lo.z - p.z, p.z - b.hi.z));
  return fmaf(gx, gx, fmaf(gy, gy, gz * gz)) <= reach * reach;
}

// a box moved by an offset (one rounding per bound, within the culling slack)
__device__ __forceinline__ Box3 box_shift(const Box3& b, float3 d) {
  Box3 r;
  r.lo = make_float3(b.lo.x + d.x, b.lo.y + d.y, b.lo.z + d.z);
  r.hi = make_float3(b.hi.x + d.x, b.hi.y + d.y, b.hi.z + d.z);
  return r;
}

// upper end of the projection of a box on u
__device__ __forceinline__ float box_rhi(const Box3& b, float3 u) {
  return fmaf(u.x, u.x >= 0.0f ? b.hi.x : b.lo.x,
              fmaf(u.y, u.y >= 0.0f ? b.hi.y : b.lo.y, u.z * (u.z >= 0.0f ? b.hi.z : b.lo.z)));
}

// Box and largest H of the warp's particles that still iterate h.  In a full pass
// every particle does, and the cluster's own box and H are returned unchanged;
// in a later pass the own side needs only the neighbours of these particles.
struct ActiveBox {
  Box3 b;
  float H;
  bool any, all;   // some / every particle of the cluster iterates
};

__device__ __forceinline__ ActiveBox active_box(const DensI& I, const Box3& bi, float Hi) {
  ActiveBox a;
  const bool ia = I.valid && I.act;
  if (__all_sync(0xffffffffu, ia || !I.valid)) {
    a.b = bi;
    a.H = Hi;
    a.any = a.all = true;
    return a;
  }
  a.all = false;
  a.any = __any_sync(0xffffffffu, ia);
  a.b.lo = make_float3(warp_min(ia ? I.p.x : 1e30f), warp_min(ia ? I.p.y : 1e30f), warp_min(ia ? I.p.z : 1e30f));
  a.b.hi = make_float3(warp_max(ia ? I.p.x : -1e30f), warp_max(ia ? I.p.y : -1e30f), warp_max(ia ? I.p.z : -1e30f));
  a.H = warp_max(ia ? I.H : 0.0f);
  return a;
}

// Pair-interaction setup shared by the density and force kernels.
struct PairSetup {
  int A, B;
  ItemGeom g;
  float3 shA, shB;        // particle frame offsets: leaf frame -> A's frame (B includes e db)
  float3 tshA, tshB;      // cluster box offsets (the leaf centre is added per cluster)
  float3 u;
  unsigned int sb, ntj;   // B's sorted cluster list (sb = SORT_NONE: B's clusters in their own order)
  unsigned int tb0;       // B's first cluster
  float HmB, slack;
  Box3 cellB;             // B's cell in A's frame
};

__device__ __forceinline__ PairSetup pair_setup(const Lists& Lq, const Tree& T, const BoxDesc* box, int item) {
  PairSetup P;
  P.A = Lq.pair_a[item];
  P.B = Lq.pair_b[item];
  const int ax = Lq.pair_axis[item];
  P.g = item_geom(T, box, P.A, ax);
  const float4 cA = T.cen[P.A], cB = T.cen[P.B];
  P.shA = make_float3(-cA.x, -cA.y, -cA.z);
  P.shB = make_float3(P.g.offB.x - cB.x, P.g.offB.y - cB.y, P.g.offB.z - cB.z);
  P.tshA = P.shA;
  P.tshB = P.shB;
  P.u = axis_unit_f(ax);
  P.ntj = T.ntile[P.B];
  P.tb0 = T.tile0[P.B];
  const unsigned int sbB = T.sortbase[P.B];
  P.sb = sbB == SORT_NONE ? SORT_NONE : sbB + (unsigned int)__popc(T.axes[P.B] & ((1u << ax) - 1u)) * P.ntj;
  P.HmB = T.hmax[P.B] * P.g.invL;
  P.slack = P.g.e * 1.52587890625e-05f + P.g.es + 1e-6f * fmaxf(P.HmB, T.hmax[P.A] * P.g.invL);   // 2^-16 e
  // B's cell, widened by the drift of particles kept in it since the build
  const float h = 0.5f * P.g.e + P.g.drift;
  P.cellB.lo = make_float3(P.g.offB.x - h, P.g.offB.y - h, P.g.offB.z - h);
  P.cellB.hi = make_float3(P.g.offB.x + h, P.g.offB.y + h, P.g.offB.z + h);
  return P;
}

// The frame of a pair task's particle arithmetic: the centre of the own cluster's
// leaf.  A pair of large cells that cannot split (one particle of large H in it
// is enough) still holds particles of small H; in A's frame their positions
// would be rounded at A's scale, in their leaf's frame at the leaf's.  The own
// offsets are used as stored (sh_own = -leaf centre cancels their leaf centre
// exactly), B's particles move by the exact dyadic offset sh_part, so each
// position is rounded once, at most at A's scale: the guard band stays valid.
// d: the leaf centre in A's frame (exact), for moving boxes between the frames.
struct LeafFrame {
  float3 sh_own, sh_part, d;
};

__device__ __forceinline__ LeafFrame leaf_frame(const Tiles& TL, const Tree& T, unsigned int ti, const PairSetup& P) {
  const float4 cl = TL.cen[ti], ca = T.cen[P.A];
  LeafFrame F;
  F.sh_own = make_float3(-cl.x, -cl.y, -cl.z);
  F.d = make_float3(cl.x - ca.x, cl.y - ca.y, cl.z - ca.z);
  F.sh_part = make_float3(P.shB.x - F.d.x, P.shB.y - F.d.y, P.shB.z - F.d.z);
  return F;
}

// Lane-parallel scan of B's sorted cluster list for the i cluster (box bi,
// largest support Hi): returns in *jt, *jn, *js the lane's candidate cluster,
// its size and first particle, and a ballot of the lanes whose cluster is in
// reach (sorted window, then box distance).
// *stop is set when the sorted window has passed every cluster of B.
template <bool DENS>
__device__ __forceinline__ unsigned int scan_clusters(const PairSetup& P, const Tree& T, const Tiles& TL,
                                                      const float* __restrict__ sort_r,
                                                      const unsigned int* __restrict__ sort_i, unsigned int e0,
                                                      const Box3& bi, float rhi_i, float Hi, const ActiveBox& A,
                                                      unsigned int* jt, unsigned int* jn, unsigned int* js,
                                                      bool* stop) {
  const int lane = threadIdx.x & 31;
  const bool sorted = P.sb != SORT_NONE;
  if (sorted) {
    // sort keys are the projections at the build; a cluster's projection has
    // since moved by at most the drift
    const float r0 = sort_r[P.sb + e0] + P.g.offBp - P.g.drift;
    *stop = r0 - rhi_i > fmaxf(Hi, P.HmB) + P.slack;     // the sorted list only moves further away
    if (*stop) return 0u;
  } else {
    *stop = false;
  }
  const unsigned int e = e0 + lane;
  bool pass = false;
  unsigned int t = 0;
  if (e < P.ntj) {
    t = sorted ? sort_i[P.sb + e] : P.tb0 + e;
    const float Hj = TL.lo[t].w * P.g.invL;
    const float reach = fmaxf(Hi, Hj) + P.slack;
    const bool window = !sorted || sort_r[P.sb + e] + P.g.offBp - P.g.drift - rhi_i <= reach;
    if (window) {
      const Box3 bj = tile_box3(TL, T, t, P.tshB);
      if (DENS) {
        // the neighbours of the particles that iterate, and the clusters that
        // iterate near any particle of this one
        // (with every particle iterating, the first test covers the second)
        pass = (A.any && box_near(A.b, bj, fmaxf(A.H, Hj) + P.slack)) ||
               (!A.all && TL.active[t] && box_near(bi, bj, Hj + P.slack));
      } else {
        pass = box_near(bi, bj, reach);
      }
    }
  }
  *jt = t;
  *jn = pass ? TL.n[t] : 0u;
  *js = pass ? TL.start[t] : 0u;
  return __ballot_sync(0xffffffffu, pass);
}

// One pair task: cluster ti of cell A against the sorted clusters of cell B.
template <bool COUNT, bool PART, bool KAHAN, bool REC>
__device__ __forceinline__ void density_pair_task(int item, unsigned int ti, const Lists& Lq, const Tree& T, const Tiles& TL, const BoxDesc* __restrict__ box,
    const float4* __restrict__ pos4, const float4* __restrict__ cen4, const float* __restrict__ sort_r,
    const unsigned int* __restrict__ sort_i, const unsigned char* __restrict__ act,
    const unsigned int* __restrict__ perm, const double* __restrict__ x, float4* dacc, unsigned int* dcnt, DensShared& S,
    Counters& C, const PairRec& R, RecW& W) {
  const int lane = threadIdx.x & 31;
  const PairSetup P = pair_setup(Lq, T, box, item);
  if (REC) rec_task_begin(S, Lq.p_toff[item] + (ti - T.tile0[P.A]));
  const LeafFrame F = leaf_frame(TL, T, ti, P);
  const Box3 bi = tile_box3(TL, T, ti, P.tshA);          // the cluster in A's frame (the sorted sweep)
  const Box3 bil = tile_box3(TL, T, ti, F.sh_own);       // ... and in its leaf's frame (the particles)
  const float Hi = TL.lo[ti].w * P.g.invL;
  const float rhi_i = box_rhi(bi, P.u);
  const unsigned int ni = TL.n[ti];
  const bool vi = (unsigned int)lane < ni;
  const unsigned char* actp = PART ? act : nullptr;
  const DensI I = load_dens(vi, TL.start[ti] + lane, F.sh_own, pos4, cen4, actp, P.g.invL, P.g.eb);
  dens_stage_own(S, lane, I);
  const ActiveBox AB = PART ? active_box(I, bil, Hi) : ActiveBox{bil, Hi, true, true};
  const ActiveBox ABc{box_shift(AB.b, F.d), AB.H, AB.any, AB.all};   // in A's frame
  DensAcc<KAHAN> acc;
  unsigned int cnt = 0, q = 0;
  for (unsigned int e0 = 0; e0 < P.ntj; e0 += 32) {
    unsigned int jt, jn, js;
    bool stop;
    unsigned int mask =
        scan_clusters<true>(P, T, TL, sort_r, sort_i, e0, bi, rhi_i, Hi, ABc, &jt, &jn, &js, &stop);
    if (stop) break;
    // the loads of the next candidate cluster are issued before the current
    // one is tested, so that their latency overlaps that work
    bool nv = false;
    unsigned int ng = 0;
    DensRaw nr;
    if (mask) {
      const int k = __ffs(mask) - 1;
      nv = (unsigned int)lane < __shfl_sync(0xffffffffu, jn, k);
      ng = __shfl_sync(0xffffffffu, js, k) + lane;
      nr = fetch_dens(nv, ng, pos4, cen4, actp);
    }
    while (mask) {
      mask &= mask - 1;
      const bool vj = nv;
      const unsigned int gj = ng;
      const DensRaw cr = nr;
      if (mask) {
        const int k = __ffs(mask) - 1;
        nv = (unsigned int)lane < __shfl_sync(0xffffffffu, jn, k);
        ng = __shfl_sync(0xffffffffu, js, k) + lane;
        nr = fetch_dens(nv, ng, pos4, cen4, actp);
      }
      const DensI J = make_dens(vj, gj, cr, F.sh_part, P.g.invL, P.g.eb);
      // stage only the partners within reach: of the particles that iterate (own
      // side), or, when the partner iterates, of any particle of the cluster
      const bool pass = vj && ((AB.any && near_box(J.p, AB.b, fmaxf(AB.H, J.H) + P.slack)) ||
                               (!AB.all && J.act && near_box(J.p, bil, J.H + P.slack)));
      const unsigned int bal = __ballot_sync(0xffffffffu, pass);
      const unsigned int np = __popc(bal);
      if (q + np > 32u) {
        dens_batch<COUNT, PART, KAHAN, REC>(I, S, q, false, acc, cnt, perm, x, P.g, dacc, dcnt, C, R, W);
        q = 0;
      }
      if (pass) dens_put(S, (int)(q + __popc(bal & ((1u << lane) - 1u))), J);
      q += np;
    }
  }
  if (q) dens_batch<COUNT, PART, KAHAN, REC>(I, S, q, false, acc, cnt, perm, x, P.g, dacc, dcnt, C, R, W);
  flush_dens(I.g, acc.total(), cnt, dacc, dcnt);
  if (REC) rec_task_end(R.ptask, S);
}

// One self task: cluster ti against itself and the later clusters of its cell.
template <bool COUNT, bool PART, bool KAHAN, bool REC>
__device__ __forceinline__ void density_self_task(int item, unsigned int ti, const Lists& Lq, const Tree& T, const Tiles& TL, const BoxDesc* __restrict__ box,
    const float4* __restrict__ pos4, const float4* __restrict__ cen4, const float* __restrict__ sort_r,
    const unsigned int* __restrict__ sort_i, const unsigned char* __restrict__ act,
    const unsigned int* __restrict__ perm, const double* __restrict__ x, float4* dacc, unsigned int* dcnt, DensShared& S,
    Counters& C, const PairRec& R, RecW& W) {
  const int lane = threadIdx.x & 31;
  const int A = Lq.self_a[item];
  if (REC) rec_task_begin(S, Lq.s_toff[item] + (ti - T.tile0[A]));
  const ItemGeom g = item_geom(T, box, A, 0);
  const float4 cA = T.cen[A];
  const float3 sh = make_float3(-cA.x, -cA.y, -cA.z);
  const float slack = g.e * 1.52587890625e-05f + g.es + 1e-6f * T.hmax[A] * g.invL;
  const unsigned int t0 = T.tile0[A], nt = T.ntile[A];
  const Box3 bi = tile_box3(TL, T, ti, sh);
  const float Hi = TL.lo[ti].w * g.invL;
  const bool vi = (unsigned int)lane < TL.n[ti];
  const unsigned char* actp = PART ? act : nullptr;
  const DensI I = load_dens(vi, TL.start[ti] + lane, sh, pos4, cen4, actp, g.invL, g.eb);
  dens_stage_own(S, lane, I);
  const ActiveBox AB = PART ? active_box(I, bi, Hi) : ActiveBox{bi, Hi, true, true};
  DensAcc<KAHAN> acc;
  unsigned int cnt = 0, q = 0;
  // inside the cluster itself each unordered pair once: partners above the lane
  if (vi) dens_put(S, lane, I);
  dens_batch<COUNT, PART, KAHAN, REC>(I, S, TL.n[ti], true, acc, cnt, perm, x, g, dacc, dcnt, C, R, W);
  // the later clusters of the cell, 32 box tests at a time
  for (unsigned int b0 = ti + 1; b0 < t0 + nt; b0 += 32) {
    const unsigned int tl = b0 + lane;
    bool ok = false;
    if (tl < t0 + nt) {
      const Box3 bj = tile_box3(TL, T, tl, sh);
      const float Hj = TL.lo[tl].w * g.invL;
      ok = (AB.any && box_near(AB.b, bj, fmaxf(AB.H, Hj) + slack)) ||
           (!AB.all && TL.active[tl] && box_near(bi, bj, Hj + slack));
    }
    unsigned int mask = __ballot_sync(0xffffffffu, ok);
    while (mask) {
      const int k = __ffs(mask) - 1;
      mask &= mask - 1;
      const unsigned int tj = b0 + (unsigned int)k;
      const bool vj = (unsigned int)lane < TL.n[tj];
      const DensI J = load_dens(vj, TL.start[tj] + lane, sh, pos4, cen4, actp, g.invL, g.eb);
      const bool pass = vj && ((AB.any && near_box(J.p, AB.b, fmaxf(AB.H, J.H) + slack)) ||
                               (!AB.all && J.act && near_box(J.p, bi, J.H + slack)));
      const unsigned int bal = __ballot_sync(0xffffffffu, pass);
      const unsigned int np = __popc(bal);
      if (q + np > 32u) {
        dens_batch<COUNT, PART, KAHAN, REC>(I, S, q, false, acc, cnt, perm, x, g, dacc, dcnt, C, R, W);
        q = 0;
      }
      if (pass) dens_put(S, (int)(q + __popc(bal & ((1u << lane) - 1u))), J);
      q += np;
    }
  }
  if (q) dens_batch<COUNT, PART, KAHAN, REC>(I, S, q, false, acc, cnt, perm, x, g, dacc, dcnt, C, R, W);
  flush_dens(I.g, acc.total(), cnt, dacc, dcnt);
  if (REC) rec_task_end(R.stask, S);
}

template <bool COUNT>
__device__ __forceinline__ void force_pair_task(int item, unsigned int ti, const Lists& Lq, const Tree& T, const Tiles& TL, const BoxDesc* __restrict__ box,
    const float4* __restrict__ pos4, const float4* __restrict__ cen4, const float4* __restrict__ vel4,
    const float4* __restrict__ ghost4, const float* __restrict__ sort_r, const unsigned int* __restrict__ sort_i,
    const unsigned int* __restrict__ perm, const double* __restrict__ x, float alpha, float4* facc, float* fvsig,
    unsigned int* fcnt, ForceShared& S, Counters* C) {
  const int lane = threadIdx.x & 31;
  const PairSetup P = pair_setup(Lq, T, box, item);
  const LeafFrame F = leaf_frame(TL, T, ti, P);
  const Box3 bi = tile_box3(TL, T, ti, P.tshA);          // the cluster in A's frame (the sorted sweep)
  const Box3 bil = tile_box3(TL, T, ti, F.sh_own);       // ... and in its leaf's frame (the particles)
  const float Hi = TL.lo[ti].w * P.g.invL;
  const float rhi_i = box_rhi(bi, P.u);
  const bool vi = (unsigned int)lane < TL.n[ti];
  const ForceI I = load_force(vi, TL.start[ti] + lane, F.sh_own, pos4, cen4, vel4, ghost4, P.g.invL, P.g.L32, P.g.eb);
  force_stage_own(S, lane, I);
  unsigned int q = 0;
  for (unsigned int e0 = 0; e0 < P.ntj; e0 += 32) {
    unsigned int jt, jn, js;
    bool stop;
    unsigned int mask =
        scan_clusters<false>(P, T, TL, sort_r, sort_i, e0, bi, rhi_i, Hi, ActiveBox{bi, Hi, true, true}, &jt, &jn, &js,
                             &stop);
    if (stop) break;
    while (mask) {
      const int k = __ffs(mask) - 1;
      mask &= mask - 1;
      const bool vj = (unsigned int)lane < __shfl_sync(0xffffffffu, jn, k);
      const ForceI J = load_force(vj, __shfl_sync(0xffffffffu, js, k) + lane, F.sh_part, pos4, cen4, vel4, ghost4,
                                  P.g.invL, P.g.L32, P.g.eb);
      const bool pass = vj && near_box(J.p, bil, fmaxf(Hi, J.H) + P.slack);
      const unsigned int bal = __ballot_sync(0xffffffffu, pass);
      const unsigned int np = __popc(bal);
      if (q + np > 32u) {
        force_batch<COUNT>(S, q, false, perm, x, box_exact(P.g), alpha, facc, fvsig, fcnt, C);
        q = 0;
      }
      if (pass) force_put(S, (int)(q + __popc(bal & ((1u << lane) - 1u))), J);
      q += np;
    }
  }
  if (q) force_batch<COUNT>(S, q, false, perm, x, box_exact(P.g), alpha, facc, fvsig, fcnt, C);
  __syncwarp();
  flush_force(__float_as_int(S.ih[lane].w), S.iacc[lane], S.ivs[lane], facc, fvsig);
}

template <bool COUNT>
__device__ __forceinline__ void force_self_task(int item, unsigned int ti, const Lists& Lq, const Tree& T, const Tiles& TL, const BoxDesc* __restrict__ box,
    const float4* __restrict__ pos4, const float4* __restrict__ cen4, const float4* __restrict__ vel4,
    const float4* __restrict__ ghost4, const float* __restrict__ sort_r, const unsigned int* __restrict__ sort_i,
    const unsigned int* __restrict__ perm, const double* __restrict__ x, float alpha, float4* facc, float* fvsig,
    unsigned int* fcnt, ForceShared& S, Counters* C) {
  const int lane = threadIdx.x & 31;
  const int A = Lq.self_a[item];
  const ItemGeom g = item_geom(T, box, A, 0);
  const float4 cA = T.cen[A];
  const float3 sh = make_float3(-cA.x, -cA.y, -cA.z);
  const float slack = g.e * 1.52587890625e-05f + g.es + 1e-6f * T.hmax[A] * g.invL;
  const unsigned int t0 = T.tile0[A], nt = T.ntile[A];
  const Box3 bi = tile_box3(TL, T, ti, sh);
  const float Hi = TL.lo[ti].w * g.invL;
  const bool vi = (unsigned int)lane < TL.n[ti];
  const ForceI I = load_force(vi, TL.start[ti] + lane, sh, pos4, cen4, vel4, ghost4, g.invL, g.L32, g.eb);
  force_stage_own(S, lane, I);
  unsigned int q = 0;
  // inside the cluster itself each unordered pair once: partners above the lane
  if (vi) force_put(S, lane, I);
  force_batch<COUNT>(S, TL.n[ti], true, perm, x, box_exact(g), alpha, facc, fvsig, fcnt, C);
  for (unsigned int b0 = ti + 1; b0 < t0 + nt; b0 += 32) {
    const unsigned int tl = b0 + lane;
    bool ok = false;
    if (tl < t0 + nt) {
      const Box3 bj = tile_box3(TL, T, tl, sh);
      ok = box_near(bi, bj, fmaxf(Hi, TL.lo[tl].w * g.invL) + slack);
    }
    unsigned int mask = __ballot_sync(0xffffffffu, ok);
    while (mask) {
      const int k = __ffs(mask) - 1;
      mask &= mask - 1;
      const unsigned int tj = b0 + (unsigned int)k;
      const bool vj = (unsigned int)lane < TL.n[tj];
      const ForceI J = load_force(vj, TL.start[tj] + lane, sh, pos4, cen4, vel4, ghost4, g.invL, g.L32, g.eb);
      const bool pass = vj && near_box(J.p, bi, fmaxf(Hi, J.H) + slack);
      const unsigned int bal = __ballot_sync(0xffffffffu, pass);
      const unsigned int np = __popc(bal);
      if (q + np > 32u) {
        force_batch<COUNT>(S, q, false, perm, x, box_exact(g), alpha, facc, fvsig, fcnt, C);
        q = 0;
      }
      if (pass) force_put(S, (int)(q + __popc(bal & ((1u << lane) - 1u))), J);
      q += np;
    }
  }
  if (q) force_batch<COUNT>(S, q, false, perm, x, box_exact(g), alpha, facc, fvsig, fcnt, C);
  __syncwarp();
  flush_force(__float_as_int(S.ih[lane].w), S.iacc[lane], S.ivs[lane], facc, fvsig);
}

// Whether a task's records still hold when its partner cell (the own cell for a
// self task) holds particles that took a new h after the recording: they do when
// every such particle lies out of reach of the own cluster, reach taken with the
// largest H the cell has had since the recording (cell H maxima only grow within
// a step), so that no pair with them was recorded or is missing.
__device__ __forceinline__ bool changed_out_of_reach(bool self, int item, unsigned int ti, const Lists& Lq,
                                                  const Tree& T, const Tiles& TL, const BoxDesc* __restrict__ box) {
  int C;
  Box3 bi;
  float reach;
  float3 off;
  if (self) {
    C = Lq.self_a[item];
    const ItemGeom g = item_geom(T, box, C, 0);
    const float4 cA = T.cen[C];
    bi = tile_box3(TL, T, ti, make_float3(-cA.x, -cA.y, -cA.z));
    const float Hm = T.hmax[C] * g.invL;
    reach = fmaxf(TL.lo[ti].w * g.invL, Hm) + g.e * 1.52587890625e-05f + g.es + 1e-6f * Hm;
    off = make_float3(0.0f, 0.0f, 0.0f);
  } else {
    const PairSetup P = pair_setup(Lq, T, box, item);
    C = P.B;
    bi = tile_box3(TL, T, ti, P.tshA);
    reach = fmaxf(TL.lo[ti].w * P.g.invL, P.HmB) + P.slack;
    off = P.g.offB;
  }
  Box3 cb;
  cb.lo = make_float3(key_float(T.clo[3 * C]) + off.x, key_float(T.clo[3 * C + 1]) + off.y,
                      key_float(T.clo[3 * C + 2]) + off.z);
  cb.hi = make_float3(key_float(T.chi[3 * C]) + off.x, key_float(T.chi[3 * C + 1]) + off.y,
                      key_float(T.chi[3 * C + 2]) + off.z);
  return !box_near(bi, cb, reach);
}

// A force task replayed from the records of the first density pass: the frames
// of the particle arithmetic are those of force_pair_task / force_self_task, the
// batches follow the recording warp's chain of chunks.  Valid while no particle of
// the own cluster or of the partner cell (the own cell for a self task) has taken
// a new h since the recording: the recorded pairs are then the pairs at the
// current h.
template <bool COUNT>
__device__ __forceinline__ void force_replay_task(bool self, int item, unsigned int ti, uint2 rec, const PairRec& R,
    const Lists& Lq, const Tree& T, const Tiles& TL, const BoxDesc* __restrict__ box,
    const float4* __restrict__ pos4, const float4* __restrict__ cen4, const float4* __restrict__ vel4,
    const float4* __restrict__ ghost4, float alpha, float4* facc, float* fvsig, unsigned int* fcnt, ForceShared& S,
    Counters* C) {
  const int lane = threadIdx.x & 31;
  ItemGeom g;
  float3 sh_own, sh_part;
  if (self) {
    const int A = Lq.self_a[item];
    g = item_geom(T, box, A, 0);
    const float4 cA = T.cen[A];
    sh_own = make_float3(-cA.x, -cA.y, -cA.z);
    sh_part = sh_own;
  } else {
    // as pair_setup and leaf_frame
    const int A = Lq.pair_a[item], Bc = Lq.pair_b[item];
    g = item_geom(T, box, A, Lq.pair_axis[item]);
    const float4 cA = T.cen[A], cB = T.cen[Bc], cl = TL.cen[ti];
    const float3 shB = make_float3(g.offB.x - cB.x, g.offB.y - cB.y, g.offB.z - cB.z);
    const float3 d = make_float3(cl.x - cA.x, cl.y - cA.y, cl.z - cA.z);
    sh_own = make_float3(-cl.x, -cl.y, -cl.z);
    sh_part = make_float3(shB.x - d.x, shB.y - d.y, shB.z - d.z);
  }
  const bool vi = (unsigned int)lane < TL.n[ti];
  const ForceI I = load_force(vi, TL.start[ti] + lane, sh_own, pos4, cen4, vel4, ghost4, g.invL, g.L32, g.eb);
  force_stage_own(S, lane, I);
  unsigned int b = rec.x;
  for (unsigned int k = 0; k < rec.y; ++k, ++b) {
    if (k > 0 && b % REC_CHUNK == 0u) b = R.next[b / REC_CHUNK - 1u] * REC_CHUNK;   // the chunk is full: next one
    const bool own_only = self && k == 0;
    if (own_only) {
      __syncwarp();
      if (vi) force_put(S, lane, I);
    }
    force_replay_batch<COUNT>(S, R.pool + 64ull * b, own_only, sh_part, g.invL, g.L32, g.eb, pos4, cen4, vel4,
                              ghost4, alpha, facc, fvsig, fcnt, C);
  }
  __syncwarp();
  flush_force(__float_as_int(S.ih[lane].w), S.iacc[lane], S.ivs[lane], facc, fvsig);
}

// Density interactions of one pass: the live pair and self tasks in one queue.
// PART: a later pass of the h iteration (particles still iterating), where the own
// side culls against the box of the cluster's iterating particles; the first pass
// (every particle) has its own instance without that code.  Both are launched in
// a captured step, and the one that does not match the iteration returns.
// The first pass (PART = false) runs 7 blocks of 128 threads per SM (at most 73
// registers, a few spilled): the pass waits mostly on partner loads, and more warps
// in flight hide more of them (33.5M: 62.8 ms at 5 blocks, 61.5 at 6, 60.5 at 7,
// 61.7 at 8, where the spills grow).
template <bool COUNT, bool PART, bool KAHAN, bool REC>
__global__ void __launch_bounds__(SPH_THREADS, PART ? PART_BLOCKS : (REC ? REC_BLOCKS : DENS_BLOCKS)) k_density(Lists Lq, Tree T, Tiles TL, const BoxDesc* __restrict__ box,
                                                         const float4* __restrict__ pos4,
                                                         const float4* __restrict__ cen4,
                                                         const float* __restrict__ sort_r,
                                                         const unsigned int* __restrict__ sort_i,
                                                         const unsigned char* __restrict__ act,
                                                         const unsigned int* __restrict__ perm,
                                                         const double* __restrict__ x, float4* dacc,
                                                         unsigned int* dcnt, unsigned long long* pc,
                                                         unsigned int* __restrict__ task_ctr, int partial_host,
                                                         const int* __restrict__ it_dev, const int* __restrict__ gflag,
                                                         const unsigned int* __restrict__ g_n, unsigned int cap_g,
                                                         const __grid_constant__ PairRec Rec) {
  pdl_wait();
  const int partial = it_dev ? (*it_dev > 1 ? 1 : 0) : partial_host;
  if ((partial != 0) != PART) return;
  if (PART && gflag && gather_on(gflag, g_n, cap_g)) return;   // the pass gathers
  __shared__ DensShared SH[SPH_WARPS_PER_CTA];
  const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  DensShared& S = SH[wl];
  RecW W;
  Counters Cp, Cs;
  const unsigned int ntask = *Lq.n_live;
  // few tasks (the later passes of the h iteration): one task per fetch and no
  // fetch ahead, so that no warp queues several while others idle
  const bool few = ntask < 4u * gridDim.x * (blockDim.x >> 5);
  // (8 at a time only where every warp gets many: smaller passes keep their balance)
  const unsigned int chunk = few ? 1u : (ntask >= 64u * gridDim.x * (blockDim.x >> 5) ? TASK_CHUNK_DENSITY : 2u);
  unsigned int raw = 0;
  if (lane == 0) raw = atomicAdd(task_ctr, chunk);
  for (unsigned int base = __shfl_sync(0xffffffffu, raw, 0); base < ntask; base = __shfl_sync(0xffffffffu, raw, 0)) {
    if (!few && lane == 0) raw = atomicAdd(task_ctr, chunk);    // the next chunk, fetched while this one runs
    const unsigned int tend = min(base + chunk, ntask);
    for (unsigned int t = base; t < tend; ++t) {
      const uint2 lt = Lq.p_live[t];
      const int item = (int)(lt.x & 0x7fffffffu);
      if (lt.x >> 31)
        density_self_task<COUNT, PART, KAHAN, REC && !PART>(item, lt.y, Lq, T, TL, box, pos4, cen4, sort_r, sort_i, act,
                                                       perm, x, dacc, dcnt, S, Cs, Rec, W);
      else
        density_pair_task<COUNT, PART, KAHAN, REC && !PART>(item, lt.y, Lq, T, TL, box, pos4, cen4, sort_r, sort_i, act,
                                                       perm, x, dacc, dcnt, S, Cp, Rec, W);
    }
    if (few && lane == 0) raw = atomicAdd(task_ctr, chunk);
  }
  commit_counters<COUNT>(Cp, pc, 0);
  commit_counters<COUNT>(Cs, pc, 1);
}

// Force interactions of one pass: the pair and self tasks in one queue.
// Registers capped at 64 per thread (8 blocks of 128 threads, whose shared memory
// fits an SM with the 768-entry pair list): more warps in flight to hide the
// partner loads outweigh the few spilled values (33.5M: 6, 5 and 4 blocks took 74,
// 84 and 98 ms against 65 ms).
template <bool COUNT>
__global__ void __launch_bounds__(SPH_THREADS, 8) k_force(Lists Lq, Tree T, Tiles TL, const BoxDesc* __restrict__ box,
                                                       const float4* __restrict__ pos4,
                                                       const float4* __restrict__ cen4,
                                                       const float4* __restrict__ vel4,
                                                       const float4* __restrict__ ghost4,
                                                       const float* __restrict__ sort_r,
                                                       const unsigned int* __restrict__ sort_i,
                                                       const unsigned int* __restrict__ perm,
                                                       const double* __restrict__ x, float alpha, float4* facc,
                                                       float* fvsig, unsigned int* fcnt, unsigned long long* pc,
                                                       unsigned int* __restrict__ task_ctr,
                                                       const __grid_constant__ PairRec R) {
  pdl_wait();
  __shared__ ForceShared SH[SPH_WARPS_PER_CTA];
  const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  ForceShared& S = SH[wl];
  Counters Cp, Cs;
  const unsigned int ntask = *Lq.n_live;
  // few tasks (the later passes of the h iteration): one task per fetch and no
  // fetch ahead, so that no warp queues several while others idle
  const bool few = ntask < 4u * gridDim.x * (blockDim.x >> 5);
  const unsigned int chunk = few ? 1u : TASK_CHUNK_FORCE;
  unsigned int raw = 0;
  if (lane == 0) raw = atomicAdd(task_ctr, chunk);
  for (unsigned int base = __shfl_sync(0xffffffffu, raw, 0); base < ntask; base = __shfl_sync(0xffffffffu, raw, 0)) {
    if (!few && lane == 0) raw = atomicAdd(task_ctr, chunk);    // the next chunk, fetched while this one runs
    const unsigned int tend = min(base + chunk, ntask);
    for (unsigned int t = base; t < tend; ++t) {
      const uint2 lt = Lq.p_live[t];
      const int item = (int)(lt.x & 0x7fffffffu);
      const bool self = (lt.x >> 31) != 0u;
      // the records of the first density pass, where they hold
      uint2 rec = make_uint2(REC_NONE, 0u);
      if (R.pool && !TL.changed[lt.y]) {
        const int A = self ? Lq.self_a[item] : Lq.pair_a[item];
        const int C = self ? A : Lq.pair_b[item];
        if (!T.changed[C] || changed_out_of_reach(self, item, lt.y, Lq, T, TL, box))
          rec = self ? R.stask[Lq.s_toff[item] + (lt.y - T.tile0[A])] : R.ptask[Lq.p_toff[item] + (lt.y - T.tile0[A])];
      }
      if (COUNT && lane == 0) atomicAdd(&pc[rec.x != REC_NONE ? 11 : 12], 1ull);
      if (rec.x != REC_NONE)
        force_replay_task<COUNT>(self, item, lt.y, rec, R, Lq, T, TL, box, pos4, cen4, vel4, ghost4, alpha, facc,
                                 fvsig, fcnt, S, COUNT ? (self ? &Cs : &Cp) : nullptr);
      else if (self)
        force_self_task<COUNT>(item, lt.y, Lq, T, TL, box, pos4, cen4, vel4, ghost4, sort_r, sort_i, perm, x, alpha,
                               facc, fvsig, fcnt, S, COUNT ? &Cs : nullptr);
      else
        force_pair_task<COUNT>(item, lt.y, Lq, T, TL, box, pos4, cen4, vel4, ghost4, sort_r, sort_i, perm, x, alpha,
                               facc, fvsig, fcnt, S, COUNT ? &Cp : nullptr);
    }
    if (few && lane == 0) raw = atomicAdd(task_ctr, chunk);
  }
  commit_counters<COUNT>(Cp, pc, 2);
  commit_counters<COUNT>(Cs, pc, 3);
}





// Tasks of one pass that have work, as (interaction, cluster); bit 31 of the
// interaction marks a self task.  Pair tasks: in a density pass those whose
// cluster or partner cell still iterates h, and in every pass those whose
// cluster lies within reach of the partner cell (the test the sweep would
// start with).  Self tasks: in a density pass those whose cell still iterates
// h.  Self tasks come first: the costliest tasks are then taken early and the
// short pair tasks fill the end of the pass.  One thread per task;
// warp-aggregated appends.
template <bool DENS>
__global__ void k_live_tasks(Lists Lq, Tree T, Tiles TL, const BoxDesc* __restrict__ box, long long npt,
                             long long nst, int partial_host, const int* __restrict__ it_dev, int cap_p, int cap_s,
                             const int* __restrict__ gflag, const unsigned int* __restrict__ g_n,
                             unsigned int cap_g) {
  pdl_wait();
  const int lane = threadIdx.x & 31;
  if (it_dev && it_dev[2] != 0) return;    // the iteration has stopped: no tasks
  if (npt < 0) {
    // a captured step: the task counts of this build, from the device
    npt = min(Lq.counts[6], cap_p);
    nst = min(Lq.counts[7], cap_s);
  }
  // later iterations keep only what still iterates (with a device counter: from iteration 2 on)
  const int partial = it_dev ? (*it_dev > 1 ? 1 : 0) : partial_host;
  if (DENS && partial && gflag && gather_on(gflag, g_n, cap_g)) return;   // the pass gathers
  const long long ntask = npt + nst;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long b0 = (long long)blockIdx.x * blockDim.x; b0 < ntask; b0 += stride) {
    const long long t = b0 + threadIdx.x;
    bool live = false;
    unsigned int rec = 0, ti = 0;
    if (t < nst) {
      const unsigned int ts = (unsigned int)t;
      const int item = (int)Lq.s_task[ts];
      const int A = Lq.self_a[item];
      ti = T.tile0[A] + (ts - Lq.s_toff[item]);
      rec = (unsigned int)item | 0x80000000u;
      live = !DENS || T.active[A];
    } else if (t < ntask) {
      const unsigned int tp = (unsigned int)(t - nst);
      const int item = (int)Lq.p_task[tp];
      const int A0 = Lq.pair_a[item], B0 = Lq.pair_b[item];
      ti = T.tile0[A0] + (tp - Lq.p_toff[item]);
      rec = (unsigned int)item;
      const bool iact = !DENS || partial == 0 || TL.active[ti];
      live = iact || T.active[B0];
      if (live) {
        const PairSetup P = pair_setup(Lq, T, box, item);
        const Box3 bi = tile_box3(TL, T, ti, P.tshA);
        const float Hi = TL.lo[ti].w * P.g.invL;
        live = box_near(bi, P.cellB, fmaxf(Hi, P.HmB) + P.slack);
        if (live && !iact) {
          // only B's active particles need this cluster: their box, in A's frame,
          // must lie within B's largest H
          Box3 ba;
          ba.lo = make_float3(key_float(T.alo[3 * B0]) + P.g.offB.x, key_float(T.alo[3 * B0 + 1]) + P.g.offB.y,
                              key_float(T.alo[3 * B0 + 2]) + P.g.offB.z);
          ba.hi = make_float3(key_float(T.ahi[3 * B0]) + P.g.offB.x, key_float(T.ahi[3 * B0 + 1]) + P.g.offB.y,
                              key_float(T.ahi[3 * B0 + 2]) + P.g.offB.z);
          live = box_near(bi, ba, P.HmB + P.slack);
        }
      }
    }
    const unsigned int bal = __ballot_sync(0xffffffffu, live);
    unsigned int at = 0;
    if (lane == 0 && bal) at = atomicAdd(Lq.n_live, (unsigned int)__popc(bal));
    at = __shfl_sync(0xffffffffu, at, 0);
    if (live) Lq.p_live[at + __popc(bal & ((1u << lane) - 1u))] = make_uint2(rec, ti);
  }
}

// =========================================================================== gathered later passes
// A later pass of the h iteration needs the density sums of the particles still
// iterating only (Section II-D: the density loop runs again for the particles
// whose h has not converged).  Tracked per cluster and cell, a few per cent of
// randomly placed iterating particles make most clusters and cells active, and
// the symmetric tasks then run nearly in full for their partner side.  A later
// pass with few iterating particles gathers instead: each leaf's iterating
// particles are packed, in their sorted order, into clusters of up to 32, so that
// the packed clusters of a cell are one range; every interaction then runs once
// per packed cluster of each of its cells, the own side only — for a pair (A, B)
// A's packed clusters against B's clusters and B's against A's, for the self
// interaction of A its packed clusters against all of A's clusters with the
// particle itself left out.  A pair with r < H_i of an iterating particle i lies
// in exactly one interaction (Section II-B), and there it is taken once, from i.

// The packing runs for the later passes only (the first pass of a captured
// iteration returns at once, and so does a stopped iteration).
__device__ __forceinline__ bool later_pass(const int* it_dev) { return it_dev[0] > 1 && it_dev[2] == 0; }

// Particles still iterating per cluster (cnt[t] for the nt clusters of this
// build, and cnt[nt] = 0); clears the gathered task count.  One warp per cluster.
__global__ void k_pack_count(long long ntcap, const unsigned int* __restrict__ ntile_dev, const int* __restrict__ it_dev,
                             Tiles TL, const unsigned char* __restrict__ act, unsigned int* __restrict__ cnt,
                             unsigned int* __restrict__ g_n) {
  pdl_wait();
  if (!later_pass(it_dev)) return;
  const long long nt = ntile_dev ? min(ntcap, (long long)*ntile_dev) : ntcap;
  const int lane = threadIdx.x & 31;
  if (blockIdx.x == 0 && threadIdx.x == 0) *g_n = 0;
  const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long t = warp; t <= nt; t += nwarps) {
    bool a = false;
    if (t < nt) a = (unsigned int)lane < TL.n[t] && act[TL.start[t] + lane];
    const unsigned int c = __popc(__ballot_sync(0xffffffffu, a));
    if (lane == 0) cnt[t] = c;
  }
}

// After the scan of the counts (rank[t]: iterating particles before cluster t):
// the packed clusters of each leaf, at its first cluster (0 elsewhere).
__global__ void k_pack_leaf(long long ntcap, const unsigned int* __restrict__ ntile_dev, const int* __restrict__ it_dev,
                            Tree T, Tiles TL, const unsigned int* __restrict__ rank, unsigned int* __restrict__ v) {
  pdl_wait();
  if (!later_pass(it_dev)) return;
  const long long nt = ntile_dev ? min(ntcap, (long long)*ntile_dev) : ntcap;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t <= nt;
       t += (long long)gridDim.x * blockDim.x) {
    unsigned int val = 0;
    if (t < nt) {
      const unsigned int L = TL.leaf[t];
      if (T.tile0[L] == (unsigned int)t) val = (rank[t + T.ntile[L]] - rank[t] + 31u) >> 5;
    }
    v[t] = val;
  }
}

// The packed clusters (after the scan of k_pack_leaf's counts: pk0[t], the first
// packed cluster of the leaf whose first cluster is t): the sorted indices of the
// iterating particles by rank (idx), and per packed cluster its first rank and
// its leaf's first cluster (info) and its size (pn).  One warp per cluster.
__global__ void k_pack_fill(long long ntcap, const unsigned int* __restrict__ ntile_dev, const int* __restrict__ it_dev,
                            Tree T, Tiles TL, const unsigned char* __restrict__ act,
                            const unsigned int* __restrict__ rank, const unsigned int* __restrict__ pk0,
                            unsigned int* __restrict__ idx, uint2* __restrict__ info, unsigned char* __restrict__ pn) {
  pdl_wait();
  if (!later_pass(it_dev)) return;
  const long long nt = ntile_dev ? min(ntcap, (long long)*ntile_dev) : ntcap;
  const int lane = threadIdx.x & 31;
  const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long t = warp; t < nt; t += nwarps) {
    const unsigned int s = TL.start[t];
    const bool a = (unsigned int)lane < TL.n[t] && act[s + lane];
    const unsigned int bal = __ballot_sync(0xffffffffu, a);
    if (!bal || !a) continue;
    const unsigned int L = TL.leaf[t], t0 = T.tile0[L];
    const unsigned int r0 = rank[t0];                        // the leaf's first rank
    const unsigned int na = rank[t0 + T.ntile[L]] - r0;       // its iterating particles
    const unsigned int k = rank[t] - r0 + __popc(bal & ((1u << lane) - 1u));
    idx[r0 + k] = s + (unsigned int)lane;
    if ((k & 31u) == 0u) {
      const unsigned int pid = pk0[t0] + (k >> 5);
      info[pid] = make_uint2(r0 + k, t0);
      pn[pid] = (unsigned char)min(32u, na - k);
    }
  }
}

// The gathered tasks of a later pass, when it gathers: (interaction, packed
// cluster), bit 31 of the interaction marking a self interaction and bit 30 the
// direction of a pair (0: the packed clusters of A against B, 1: of B against
// A).  The pass gathers when it is a later one, the caller allows it and at most
// an eighth of the particles iterate (gflag[0]); the symmetric path runs instead
// when the tasks exceed the buffer.  One thread per interaction, self
// interactions first; warp-aggregated appends.
__global__ void k_gather_tasks(Lists Lq, Tree T, long long npair, long long nself, int cap_pair, int cap_self,
                               const int* __restrict__ it_dev, long long N, int allow,
                               const unsigned int* __restrict__ pk0, const unsigned int* __restrict__ pk_tot,
                               uint2* __restrict__ tasks, unsigned int* __restrict__ g_n, unsigned int cap_g,
                               int* __restrict__ gflag) {
  pdl_wait();
  const bool on = allow != 0 && later_pass(it_dev) && 8ull * pk_tot[0] <= (unsigned long long)N;
  if (blockIdx.x == 0 && threadIdx.x == 0) gflag[0] = on ? 1 : 0;
  if (!on) return;
  if (npair < 0) {
    npair = min(Lq.counts[1], cap_pair);
    nself = min(Lq.counts[0], cap_self);
  }
  const int lane = threadIdx.x & 31;
  const long long nitem = nself + npair;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long b0 = (long long)blockIdx.x * blockDim.x; b0 < nitem; b0 += stride) {
    const long long i = b0 + threadIdx.x;
    unsigned int code = 0, a0 = 0, a1 = 0, c0 = 0, c1 = 0;
    if (i < nself) {
      const int A = Lq.self_a[i];
      a0 = pk0[T.tile0[A]];
      a1 = pk0[T.tile0[A] + T.ntile[A]];
      code = (unsigned int)i | 0x80000000u;
    } else if (i < nitem) {
      const int j = (int)(i - nself);
      const int A = Lq.pair_a[j], B = Lq.pair_b[j];
      a0 = pk0[T.tile0[A]];
      a1 = pk0[T.tile0[A] + T.ntile[A]];
      c0 = pk0[T.tile0[B]];
      c1 = pk0[T.tile0[B] + T.ntile[B]];
      code = (unsigned int)j;
    }
    const unsigned int mine = (a1 - a0) + (c1 - c0);
    unsigned int incl = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    const unsigned int wtot = __shfl_sync(0xffffffffu, incl, 31);
    unsigned int base = 0;
    if (lane == 31 && wtot) base = atomicAdd(g_n, wtot);
    base = __shfl_sync(0xffffffffu, base, 31);
    unsigned int at = base + incl - mine;
    for (unsigned int p = a0; p < a1; ++p, ++at)
      if (at < cap_g) tasks[at] = make_uint2(code, p);
    for (unsigned int p = c0; p < c1; ++p, ++at)
      if (at < cap_g) tasks[at] = make_uint2(code | 0x40000000u, p);
  }
}

// r < H_i over the first n staged partners (n a multiple of 4), exact: the FP32
// test outside the guard band, FP64 inside (as pair_masks, the own radius only).
__device__ __forceinline__ unsigned int own_mask(const DensI& I, const DensShared& S, unsigned int allow, int n,
                                                 const unsigned int* perm, const double* x, const BoxExact g) {
  const float iLo = I.H2 - I.band, iHi = I.H2 + I.band;
  unsigned int m = 0, sure = 0;
  for (int s0 = n - 4; s0 >= 0; s0 -= 4) {
#pragma unroll
    for (int k = 3; k >= 0; --k) {
      const float4 J = S.p[s0 + k];
      const float dx = I.p.x - J.x, dy = I.p.y - J.y, dz = I.p.z - J.z;
      const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
      const unsigned int ai = __float_as_uint(r2 - iLo), bi = __float_as_uint(iHi - r2);   // sign: in / out
      m = __funnelshift_l(ai, m, 1);
      sure = __funnelshift_l(ai | bi, sure, 1);
    }
  }
  unsigned int u = ~sure & allow;
  while (u) {
    const int s = __ffs(u) - 1;
    u &= u - 1;
    const unsigned int bit = 1u << s;
    m = exact_less(I.g, S.g[s], I.Hphys, perm, x, g.L, g.halfL, g.periodic) ? (m | bit) : (m & ~bit);
  }
  return m & allow;
}

// One batch of q <= 32 staged partners, the own side only; in a self interaction
// the particle itself (staged with its cell) is left out.
template <bool KAHAN>
__device__ __forceinline__ void gather_batch(const DensI& I, DensShared& S, unsigned int q, bool self,
                                             DensAcc<KAHAN>& acc, unsigned int& cnt, const unsigned int* perm,
                                             const double* x, const BoxExact g) {
  const int lane = threadIdx.x & 31;
  const bool v = (unsigned int)lane < q;
  __syncwarp();
  if (!v) S.p[lane] = make_float4(1e30f, 1e30f, 1e30f, -1.0f);
  const unsigned int jvalid = __ballot_sync(0xffffffffu, v);
  __syncwarp();
  const unsigned int m = I.valid ? own_mask(I, S, jvalid, (int)((q + 3u) & ~3u), perm, x, g) : 0u;
  for (unsigned int b = m; b; b &= b - 1) {
    const int sj = __ffs(b) - 1;
    if (self && S.g[sj] == I.g) continue;
    const float4 J = S.p[sj];
    const float dx = I.p.x - J.x, dy = I.p.y - J.y, dz = I.p.z - J.z;
    dens_add(pair_r(fmaf(dz, dz, fmaf(dy, dy, dx * dx))), I.invH, S.a[sj].z, acc, cnt);
  }
  __syncwarp();
}

// One gathered task: packed cluster pid (of cell O) against the clusters of cell X.
// The frame is the packed cluster's leaf centre; X's particles move into it by
// the exact dyadic offset of the pair kernel's leaf frame (X's centre image minus
// O's centre, taken in the same order), so each position is rounded once, at
// most at the cells' scale, and the guard band holds as there.
template <bool KAHAN>
__device__ __forceinline__ void gather_task(uint2 tk, const Lists& Lq, const Tree& T, const Tiles& TL,
                                            const BoxDesc* __restrict__ box, const float4* __restrict__ pos4,
                                            const float4* __restrict__ cen4, const unsigned int* __restrict__ perm,
                                            const double* __restrict__ x, float4* dacc, unsigned int* dcnt,
                                            const uint2* __restrict__ pk_info, const unsigned char* __restrict__ pk_n,
                                            const unsigned int* __restrict__ pk_idx, DensShared& S) {
  const int lane = threadIdx.x & 31;
  const bool self = (tk.x >> 31) != 0u, dir1 = ((tk.x >> 30) & 1u) != 0u;
  const int item = (int)(tk.x & 0x3fffffffu);
  int O, X, ax = 0;
  if (self) {
    O = X = Lq.self_a[item];
  } else {
    const int A = Lq.pair_a[item], B = Lq.pair_b[item];
    ax = Lq.pair_axis[item];
    O = dir1 ? B : A;
    X = dir1 ? A : B;
  }
  // pair items join cells of one level: A's geometry serves both directions
  const ItemGeom g = item_geom(T, box, self ? O : Lq.pair_a[item], ax);
  const float3 offX = self ? make_float3(0.f, 0.f, 0.f)
                           : (dir1 ? make_float3(-g.offB.x, -g.offB.y, -g.offB.z) : g.offB);
  const uint2 info = pk_info[tk.y];
  const unsigned int n = pk_n[tk.y];
  const float4 cO = T.cen[O], cX = T.cen[X], cl = TL.cen[info.y];
  const float3 shX = make_float3(offX.x - cX.x, offX.y - cX.y, offX.z - cX.z);
  const float3 d = make_float3(cl.x - cO.x, cl.y - cO.y, cl.z - cO.z);
  const float3 sh_part = make_float3(shX.x - d.x, shX.y - d.y, shX.z - d.z);
  const float3 sh_own = make_float3(-cl.x, -cl.y, -cl.z);
  const bool vi = (unsigned int)lane < n;
  const DensI I = load_dens(vi, vi ? pk_idx[info.x + lane] : 0u, sh_own, pos4, cen4, nullptr, g.invL, g.eb);
  // the packed particles' box and largest H: the own side reaches no further
  Box3 bo;
  bo.lo = make_float3(warp_min(vi ? I.p.x : 1e30f), warp_min(vi ? I.p.y : 1e30f), warp_min(vi ? I.p.z : 1e30f));
  bo.hi = make_float3(warp_max(vi ? I.p.x : -1e30f), warp_max(vi ? I.p.y : -1e30f), warp_max(vi ? I.p.z : -1e30f));
  const float Ho = warp_max(vi ? I.H : 0.0f);
  const float slack = g.e * 1.52587890625e-05f + g.es + 1e-6f * fmaxf(T.hmax[O], T.hmax[X]) * g.invL;
  const float reach = Ho + slack;
  if (!self) {
    // X's cell, widened by the drift since the build, in this frame
    const float h = 0.5f * g.e + g.drift;
    Box3 cx;
    cx.lo = make_float3(cX.x + sh_part.x - h, cX.y + sh_part.y - h, cX.z + sh_part.z - h);
    cx.hi = make_float3(cX.x + sh_part.x + h, cX.y + sh_part.y + h, cX.z + sh_part.z + h);
    if (!box_near(bo, cx, reach)) return;
  }
  DensAcc<KAHAN> acc;
  unsigned int cnt = 0, q = 0;
  const unsigned int t0 = T.tile0[X], nt = T.ntile[X];
  for (unsigned int b0 = 0; b0 < nt; b0 += 32) {
    bool ok = false;
    if (b0 + lane < nt) ok = box_near(bo, tile_box3(TL, T, t0 + b0 + lane, sh_part), reach);
    unsigned int mask = __ballot_sync(0xffffffffu, ok);
    while (mask) {
      const int k = __ffs(mask) - 1;
      mask &= mask - 1;
      const unsigned int tj = t0 + b0 + (unsigned int)k;
      const bool vj = (unsigned int)lane < TL.n[tj];
      const DensI J = load_dens(vj, TL.start[tj] + lane, sh_part, pos4, cen4, nullptr, g.invL, g.eb);
      const bool pass = vj && near_box(J.p, bo, reach);
      const unsigned int bal = __ballot_sync(0xffffffffu, pass);
      const unsigned int np = __popc(bal);
      if (q + np > 32u) {
        gather_batch<KAHAN>(I, S, q, self, acc, cnt, perm, x, box_exact(g));
        q = 0;
      }
      if (pass) dens_put(S, (int)(q + __popc(bal & ((1u << lane) - 1u))), J);
      q += np;
    }
  }
  if (q) gather_batch<KAHAN>(I, S, q, self, acc, cnt, perm, x, box_exact(g));
  flush_dens(I.g, acc.total(), cnt, dacc, dcnt);
}

#ifndef GATHER_BLOCKS
#define GATHER_BLOCKS 8
#endif
// The gathered density pass (a later pass of the h iteration that gathers): the
// tasks of k_gather_tasks, one per fetch; g_n[1] counts the passes that gathered.
// Returns at once when the pass runs the symmetric tasks instead.
template <bool KAHAN>
__global__ void __launch_bounds__(SPH_THREADS, GATHER_BLOCKS) k_density_gather(
    Lists Lq, Tree T, Tiles TL, const BoxDesc* __restrict__ box, const float4* __restrict__ pos4,
    const float4* __restrict__ cen4, const unsigned int* __restrict__ perm, const double* __restrict__ x,
    float4* dacc, unsigned int* dcnt, const uint2* __restrict__ tasks, unsigned int* __restrict__ g_n,
    unsigned int cap_g, const int* __restrict__ gflag, const uint2* __restrict__ pk_info,
    const unsigned char* __restrict__ pk_n, const unsigned int* __restrict__ pk_idx,
    unsigned int* __restrict__ task_ctr) {
  pdl_wait();
  if (!gather_on(gflag, g_n, cap_g)) return;
  if (blockIdx.x == 0 && threadIdx.x == 0) g_n[1] += 1u;
  __shared__ DensShared SH[SPH_WARPS_PER_CTA];
  const int lane = threadIdx.x & 31;
  DensShared& S = SH[threadIdx.x >> 5];
  const unsigned int ntask = *g_n;
  unsigned int t = 0;
  if (lane == 0) t = atomicAdd(task_ctr, 1u);
  for (t = __shfl_sync(0xffffffffu, t, 0); t < ntask; t = __shfl_sync(0xffffffffu, t, 0)) {
    gather_task<KAHAN>(tasks[t], Lq, T, TL, box, pos4, cen4, perm, x, dacc, dcnt, pk_info, pk_n, pk_idx, S);
    if (lane == 0) t = atomicAdd(task_ctr, 1u);
  }
}

// =========================================================================== ghost
// mode 0: finalise every particle at its current h (one density pass);
// mode 1: one h iteration (Newton on N~ = n_ngb, bracket, clamp) for the
//         active particles, finalising those that converged or ran out.
__global__ void k_ghost(long long N, int mode, int it_host, const int* __restrict__ it_dev, int max_iter,
                        float gamma_k, float n_ngb, float tol,
                        float gamma_gas, const unsigned int* __restrict__ perm, float* __restrict__ Hs,
                        float4* __restrict__ pos4, const float4* __restrict__ cen4, const float4* __restrict__ vel4,
                        const float4* __restrict__ dacc, unsigned char* __restrict__ act, float* __restrict__ h,
                        float* __restrict__ hlo, float* __restrict__ hhi, int* __restrict__ conv,
                        const float* __restrict__ hlimp, const unsigned int* __restrict__ leaf_of, Tree T,
                        float4* __restrict__ ghost4, float4* __restrict__ hhist, int* __restrict__ n_active,
                        unsigned int* __restrict__ err_all) {
  pdl_wait();
  // the iteration number: the host's, or in a captured step the device counter
  const int it = it_dev ? *it_dev : it_host;
  if (it_dev && it_dev[2] != 0) return;    // the iteration has stopped (batched iterations)
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < N; p += (long long)gridDim.x * blockDim.x) {
    if (mode == 1 && !act[p]) continue;
    const unsigned int i = perm[p];
    const float H = Hs[p];
    const float m = cen4[p].w;
    const float4 a = dacc[p];
    const float sw = a.z + 1.0f;          // self term w(0) = 1
    const float Nw = (32.0f / 3.0f) * sw; // (4 pi / 3) H^3 n with n = (8/pi) sum w / H^3
    const float F = Nw - n_ngb;
    const bool ok = fabsf(F) <= tol * n_ngb;
    if (mode == 1 && !ok && it < max_iter) {
      const float hc = h[i];
      float lo = hlo[i], hi = hhi[i];
      if (F < 0.0f) lo = hc;
      else hi = hc;
      // dN~/dh = gamma_K (4 pi/3) H^2 (3 n - sum (3W + r W')) = -gamma_K (32/3) sum q w' / H
      const float dN = -gamma_k * (32.0f / 3.0f) * a.w / H;
      float hn = dN > 0.0f ? hc - F / dN : (F < 0.0f ? 2.0f * hc : 0.5f * hc);
      hn = fminf(fmaxf(hn, 0.5f * hc), 2.0f * hc);
      if (lo > 0.0f && isfinite(hi) && !(hn > lo && hn < hi)) hn = 0.5f * (lo + hi);
      hlo[i] = lo;
      hhi[i] = hi;
      h[i] = hn;
      const float Hn = __fmul_rn(gamma_k, hn);
      Hs[p] = Hn;
      pos4[p].w = Hn;
      if (!(Hn < hlimp[p])) atomicOr(err_all, ERR_REBUILD);
      if (Hn > H) {
        // a cell's H_max bounds its children's: the climb ends at the first cell
        // that already covers Hn
        for (int id = (int)leaf_of[p]; id >= 0; id = T.parent[id]) {
          if (T.hmax[id] >= Hn) break;
          atomic_max_pos(&T.hmax[id], Hn);
        }
      }
      {
        // one atomic for the lanes here (every particle of a first pass may iterate)
        const unsigned int am = __activemask();
        if ((threadIdx.x & 31) == __ffs(am) - 1) atomicAdd(n_active, __popc(am));
      }
      continue;
    }
    act[p] = 0;
    conv[i] = ok ? 1 : 0;
    {
      // the root of N~(h) = N_ngb one Newton step from the final h: where the next
      // step's h iteration extrapolates from
      const float hc = h[i];
      const float dN = -gamma_k * (32.0f / 3.0f) * a.w / H;
      const float hr = dN > 0.0f ? hc - F / dN : hc;
      hhist[i].x = fminf(fmaxf(hr, 0.9f * hc), 1.1f * hc);
    }
    const float ih = 1.0f / H;
    const float K3 = SPH_KNORM * ih * ih * ih;
    const float rho = K3 * (a.x + m);
    const float u = vel4[p].w;
    const float P = (gamma_gas - 1.0f) * rho * u;
    const float c = sqrtf(gamma_gas * P / rho);
    // f = [1 + h/(3 rho) d rho/dh]^-1 = 3 rho / (-sum_j m_j r W'), without cancellation;
    // 1 when no other particle lies inside the support
    const float f = a.y < 0.0f ? -3.0f * (a.x + m) / a.y : 1.0f;
    ghost4[p] = make_float4(rho, f * P / (rho * rho), c, ih);
  }
}

__global__ void k_zero_active(long long N, const unsigned char* __restrict__ act, float4* __restrict__ dacc,
                              unsigned int* __restrict__ dcnt, int all) {
  pdl_wait();
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < N; p += (long long)gridDim.x * blockDim.x) {
    if (all || act[p]) {
      dacc[p] = make_float4(0.f, 0.f, 0.f, 0.f);
      dcnt[p] = 0;
    }
  }
}

// Mark every cell that holds a particle still iterating h (and its ancestors).
// After an h iteration: the clusters and cells that still hold a particle
// iterating h (a cluster's largest H follows the H its particles took), and for
// every cell the box of those particles in the cell's
// frame.  One warp per cluster; the cluster's box of active particles is added
// to every cell on its chain with ordered-key atomics.
__global__ void k_mark_active(long long ntile, const unsigned int* __restrict__ ntile_dev,
                              const unsigned char* __restrict__ act, const float4* __restrict__ pos4, Tree T, Tiles TL) {
  pdl_wait();
  if (ntile_dev) ntile = min(ntile, (long long)*ntile_dev);   // a captured step: this build's clusters
  const int lane = threadIdx.x & 31;
  const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long t = warp; t < ntile; t += nwarps) {
    const unsigned int n = TL.n[t], s0 = TL.start[t];
    const bool a = (unsigned int)lane < n && act[s0 + lane];
    if (!__any_sync(0xffffffffu, a)) continue;
    float3 lo = make_float3(FLT_MAX, FLT_MAX, FLT_MAX), hi = make_float3(-FLT_MAX, -FLT_MAX, -FLT_MAX);
    float hm = 0.0f;
    if (a) {
      const float4 p = pos4[s0 + lane];
      lo = make_float3(p.x, p.y, p.z);
      hi = lo;
      hm = p.w;
    }
    lo.x = warp_min(lo.x); lo.y = warp_min(lo.y); lo.z = warp_min(lo.z);
    hi.x = warp_max(hi.x); hi.y = warp_max(hi.y); hi.z = warp_max(hi.z);
    // only particles that iterate change H: the cluster's largest H grows to theirs
    hm = warp_max(hm);
    if (lane != 0) continue;
    if (hm > TL.lo[t].w) TL.lo[t].w = hm;
    TL.active[t] = 1;
    TL.changed[t] = 1;
    const float4 lc = TL.cen[t];
    for (int id = (int)TL.leaf[t]; id >= 0; id = T.parent[id]) {
      T.active[id] = 1;
      T.changed[id] = 1;
      const float4 cc = T.cen[id];
      const float ox = lc.x - cc.x, oy = lc.y - cc.y, oz = lc.z - cc.z;   // exact
      atomicMin(&T.alo[3 * id], float_key(lo.x + ox));
      atomicMin(&T.alo[3 * id + 1], float_key(lo.y + oy));
      atomicMin(&T.alo[3 * id + 2], float_key(lo.z + oz));
      atomicMax(&T.ahi[3 * id], float_key(hi.x + ox));
      atomicMax(&T.ahi[3 * id + 1], float_key(hi.y + oy));
      atomicMax(&T.ahi[3 * id + 2], float_key(hi.z + oz));
      atomicMin(&T.clo[3 * id], float_key(lo.x + ox));
      atomicMin(&T.clo[3 * id + 1], float_key(lo.y + oy));
      atomicMin(&T.clo[3 * id + 2], float_key(lo.z + oz));
      atomicMax(&T.chi[3 * id], float_key(hi.x + ox));
      atomicMax(&T.chi[3 * id + 1], float_key(hi.y + oy));
      atomicMax(&T.chi[3 * id + 2], float_key(hi.z + oz));
    }
  }
}

// clusters of the i cell per interaction: the prefix of these numbers the tasks
// Tasks: one per (interaction, cluster of its first cell).  Counts per
// interaction over the whole list capacity (zero past the list), so that the
// prefix and the task totals are ready before the host reads the list sizes.
__global__ void k_task_tiles(Lists Lq, Tree T, int cap_pair, int cap_self) {
  pdl_wait();
  const int npair = min(Lq.counts[1], cap_pair), nself = min(Lq.counts[0], cap_self);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < cap_pair + cap_self; i += gridDim.x * blockDim.x) {
    if (i < cap_pair) Lq.p_toff[i] = i < npair ? T.ntile[Lq.pair_a[i]] : 0u;
    else Lq.s_toff[i - cap_pair] = i - cap_pair < nself ? T.ntile[Lq.self_a[i - cap_pair]] : 0u;
  }
}

// task -> interaction tables (one warp per interaction)
// npair < 0: the list sizes come from the device (a captured step); the tables
// hold cap_p pair tasks and cap_s self tasks, and nothing is written past them.
__global__ void k_task_items(Lists Lq, Tree T, int npair, int nself, int cap_pair, int cap_self, unsigned int cap_p,
                             unsigned int cap_s) {
  pdl_wait();
  if (npair < 0) {
    npair = min(Lq.counts[1], cap_pair);
    nself = min(Lq.counts[0], cap_self);
  }
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int i = warp; i < npair + nself; i += nwarps) {
    const bool pr = i < npair;
    const int it = pr ? i : i - npair;
    const unsigned int t0 = pr ? Lq.p_toff[it] : Lq.s_toff[it];
    const unsigned int n = T.ntile[pr ? Lq.pair_a[it] : Lq.self_a[it]];
    unsigned int* dst = pr ? Lq.p_task : Lq.s_task;
    const unsigned int cap = pr ? cap_p : cap_s;
    for (unsigned int k = lane; k < n && t0 + k < cap; k += 32) dst[t0 + k] = (unsigned int)it;
  }
}

__global__ void k_count_unconverged(long long N, const int* __restrict__ conv, int* __restrict__ out) {
  pdl_wait();
  int c = 0;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < N; p += (long long)gridDim.x * blockDim.x)
    c += conv[p] ? 0 : 1;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}

__global__ void k_set_active(long long N, unsigned char* __restrict__ act) {
  pdl_wait();
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < N; p += (long long)gridDim.x * blockDim.x)
    act[p] = 1;
}

__global__ void k_h_bracket_reset(long long N, float* __restrict__ hlo, float* __restrict__ hhi, int* __restrict__ conv) {
  pdl_wait();
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < N; p += (long long)gridDim.x * blockDim.x) {
    hlo[p] = 0.0f;
    hhi[p] = __int_as_float(0x7f800000);
    conv[p] = 0;
  }
}

// =========================================================================== captured steps
// Conditions of a step captured as a CUDA graph with conditional nodes (one
// thread each).  keep: the decomposition stays (no particle outgrew the limits).
__global__ void k_cond_keep(cudaGraphConditionalHandle keep, const unsigned int* __restrict__ reuse_flag) {
  pdl_wait();
  cudaGraphSetConditional(keep, *reuse_flag == 0u ? 1u : 0u);
}

// start of the h iteration: iteration 1 runs
__global__ void k_iter_start(cudaGraphConditionalHandle iter, int* __restrict__ it_dev) {
  pdl_wait();
  it_dev[0] = 1;
  it_dev[2] = 0;
  cudaGraphSetConditional(iter, 1u);
}

// The same control without a graph: after iteration it_dev[0], stop (it_dev[2] =
// 1: every particle finalised or the limit reached; 2: a rebuild is needed) or
// advance to the next iteration.  Kernels of later iterations launched ahead
// return at once after a stop.
__global__ void k_iter_step(int* __restrict__ it_dev, int* __restrict__ n_active,
                            const unsigned int* __restrict__ err_all, int max_iter) {
  pdl_wait();
  if (it_dev[2] != 0) return;
  const int na = *n_active;
  if (it_dev[0] == 1) it_dev[1] = na;
  if ((*err_all & ERR_REBUILD) != 0u) it_dev[2] = 2;
  else if (na == 0 || it_dev[0] >= max_iter) it_dev[2] = 1;
  else it_dev[0] += 1;
  *n_active = 0;
}

// after iteration *it_dev: another while particles still iterate, no rebuild is
// needed and the limit is not reached; the force pass follows unless a rebuild is
// needed (the host then takes over).  n_active is cleared for the next iteration.
__global__ void k_iter_next(cudaGraphConditionalHandle iter, cudaGraphConditionalHandle force, int* __restrict__ it_dev,
                            int* __restrict__ n_active, const unsigned int* __restrict__ err_all, int max_iter,
                            int* __restrict__ first_active) {
  pdl_wait();
  const bool rebuild = (*err_all & ERR_REBUILD) != 0u;
  const int na = *n_active;
  if (*it_dev == 1) *first_active = na;
  const bool more = !rebuild && na > 0 && *it_dev < max_iter;
  if (more) *it_dev += 1;
  *n_active = 0;
  it_dev[3] = (!more && !rebuild) ? 1 : 0;     // for the conditions of later force phases
  cudaGraphSetConditional(iter, more ? 1u : 0u);
  cudaGraphSetConditional(force, (!more && !rebuild) ? 1u : 0u);
}

// a condition taken from a flag in device memory (a graph node of its own)
__global__ void k_cond_set(cudaGraphConditionalHandle h, const int* __restrict__ flag) {
  cudaGraphSetConditional(h, *flag != 0 ? 1u : 0u);
}

// the displacement of every box, written into its descriptor on the device
__global__ void k_set_drift(int nbox, BoxDesc* __restrict__ box, const unsigned long long* __restrict__ dmax) {
  pdl_wait();
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nbox; b += gridDim.x * blockDim.x) {
    const double d = __longlong_as_double((long long)dmax[b]);
    box[b].drift2 = (float)(2.0 * d);
    box[b].drift_u = (float)(d * box[b].invL);
  }
}

// =========================================================================== reductions
// FP64 conservation sums per box: sum m a (3), sum m (v.a + du/dt), sum m v (3),
// sum m (v^2/2 + u).  Block row y reduces boxes y, y + gridDim.y, ...: every
// thread accumulates its particles of the box in FP64 registers, then one block
// reduction and eight atomics per box.
__global__ void __launch_bounds__(256) k_reduce(int nbox, const long long* __restrict__ boff,
                                                const BoxDesc* __restrict__ box, const unsigned int* __restrict__ perm,
                                                const float4* __restrict__ cen4, const float4* __restrict__ vel4,
                                                const float4* __restrict__ facc, double* __restrict__ red) {
  pdl_wait();
  __shared__ double part[8][8];
  for (int b = blockIdx.y; b < nbox; b += gridDim.y) {
    const long long p0 = boff[b], p1 = boff[b + 1];
    const long long nown = box[b].nown;
    double val[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (long long p = p0 + blockIdx.x * (long long)blockDim.x + threadIdx.x; p < p1;
         p += (long long)gridDim.x * blockDim.x) {
      if ((long long)perm[p] - p0 >= nown) continue;   // a halo particle: summed by its owner
      const double m = cen4[p].w;
      const float4 vv = vel4[p];
      const float4 a = facc[p];
      const double vx = vv.x, vy = vv.y, vz = vv.z;
      val[0] += m * a.x;
      val[1] += m * a.y;
      val[2] += m * a.z;
      val[3] += m * (vx * a.x + vy * a.y + vz * a.z + (double)a.w);
      val[4] += m * vx;
      val[5] += m * vy;
      val[6] += m * vz;
      val[7] += m * (0.5 * (vx * vx + vy * vy + vz * vz) + (double)vv.w);
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      double v = val[k];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) part[w][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < 8) {
      double v = 0.0;
      for (int q = 0; q < (int)(blockDim.x >> 5); ++q) v += part[q][threadIdx.x];
      atomicAdd(&red[8 * b + threadIdx.x], v);
    }
    __syncthreads();
  }
}

// =========================================================================== time stepping
// accelerations of the last force pass, kept in caller order for the next kick
__global__ void k_save_acc(long long N, const unsigned int* __restrict__ perm, const float4* __restrict__ facc,
                           float4* __restrict__ a_in) {
  pdl_wait();
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < N; p += (long long)gridDim.x * blockDim.x)
    a_in[perm[p]] = facc[p];
}

// caller-order (a, du/dt) into the saved accelerations: which = 0 sets a (n x 3), 1 sets du/dt
__global__ void k_set_acc(long long off, long long n, int which, const float* __restrict__ src,
                          float4* __restrict__ a_in) {
  pdl_wait();
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
    float4 a = a_in[off + q];
    if (which == 0) {
      a.x = src[3 * q];
      a.y = src[3 * q + 1];
      a.z = src[3 * q + 2];
    } else {
      a.w = src[q];
    }
    a_in[off + q] = a;
  }
}

void launch_set_acc(Engine& E, long long off, long long n, int which, const float* src) {
  launch_pdl(k_set_acc, E.grid(n), 256, E.st, off, n, which, src, E.a_in.p); count_launch();
}

// half kick with the box's dt: v += a dt/2, u += du/dt dt/2 (u kept >= 0)
__global__ void k_kick(long long N, const int* __restrict__ bid, const BoxDesc* __restrict__ box,
                       const float4* __restrict__ a_in, float* __restrict__ v, float* __restrict__ u) {
  pdl_wait();
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    const float hdt = (float)(0.5 * box[bid[i]].dt);
    if (hdt == 0.0f) continue;
    const float4 a = a_in[i];
    v[3 * i] += a.x * hdt;
    v[3 * i + 1] += a.y * hdt;
    v[3 * i + 2] += a.z * hdt;
    u[i] = fmaxf(u[i] + a.w * hdt, 0.0f);
  }
}

// drift in FP64 with the box's dt, wrapped into [0, L) (periodic) or clamped (open).
// The h iteration of the new step then starts from the extrapolation of the
// last roots of N~(h) = N_ngb (hhist x: this step's, written by the ghost pass;
// y, z, w: the three before) to the new time: the polynomial through them, cubic
// once four are known, with the box's weights hc, kept within 10 % of h.  A
// particle's root moves smoothly with its neighbours, so the extrapolation is
// off by a fourth-order term in dt and most particles meet the N~ tolerance in
// the first density pass.  hlev[b] counts the earlier roots a box holds (0..3); it
// restarts at 0 when the box's h is set to other values.  Without a history y, z,
// w take the current h.
__global__ void k_drift(long long N, const int* __restrict__ bid, const BoxDesc* __restrict__ box,
                        double* __restrict__ x, const float* __restrict__ v, float* __restrict__ h,
                        float4* __restrict__ hhist, const int* __restrict__ hlev) {
  pdl_wait();
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < N; p += (long long)gridDim.x * blockDim.x) {
    const int b = bid[p];
    const BoxDesc& bd = box[b];
    if (bd.dt == 0.0) continue;
    const float hc = h[p];
    float4 hh = hhist[p];
    const int lev = hlev[b];
    if (lev > 0) {
      const float* w = bd.hw[lev];
      const float hn = fmaf(w[0], hh.x, fmaf(w[1], hh.y, fmaf(w[2], hh.z, w[3] * hh.w)));
      h[p] = fminf(fmaxf(hn, 0.9f * hc), 1.1f * hc);
      hh.w = hh.z;
      hh.z = hh.y;
      hh.y = hh.x;
    } else {
      hh.y = hc;
      hh.z = hc;
      hh.w = hc;
    }
    hhist[p] = hh;
    for (int k = 0; k < 3; ++k) {
      double xn = x[3 * p + k] + (double)v[3 * p + k] * bd.dt;
      if (bd.periodic) {
        xn -= bd.L * floor(xn * bd.invL);
        if (xn >= bd.L) xn -= bd.L;
        if (xn < 0.0 || xn >= bd.L) xn = 0.0;
      } else {
        xn = fmin(fmax(xn, 0.0), nextafter(bd.L, 0.0));
      }
      x[3 * p + k] = xn;
    }
  }
}

// =========================================================================== FP32 peak
// Independent FMA chains (8 per thread) with no memory traffic between the first
// load and the final store: the FP32 pipe's throughput.  The store depends on
// every chain so the compiler keeps them.
__global__ void __launch_bounds__(256) k_fma_peak(int iters, float a, float b, float* __restrict__ out) {
  pdl_wait();
  float v[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) v[k] = (float)(threadIdx.x + k) * 1e-3f;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = fmaf(v[k], a, b);
  }
  float s = 0.0f;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += v[k];
  if (s == 12345.678f) out[blockIdx.x] = s;   // practically never: keeps the chains live
}

double measure_fp32_peak(cudaStream_t st, int nsm, float* scratch) {
  const int blocks = nsm * 8, threads = 256, iters = 8192;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  k_fma_peak<<<blocks, threads, 0, st>>>(iters, 0.9999f, 1e-4f, scratch); count_launch();
  cudaEventRecord(e0, st);
  k_fma_peak<<<blocks, threads, 0, st>>>(iters, 0.9999f, 1e-4f, scratch); count_launch();
  cudaEventRecord(e1, st);
  cudaEventSynchronize(e1);
  float ms = 0.0f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  const double flops = 2.0 * 8.0 * iters * (double)blocks * threads;
  return ms > 0.0f ? flops / (ms * 1e-3) / 1e12 : 0.0;
}

// =========================================================================== outputs
// Write field `field` of the particles of one box [off, off + n) in caller order.
__global__ void k_get_field(long long off, long long n, int field, const unsigned int* __restrict__ perm,
                            const float* __restrict__ Hs, const float4* __restrict__ cen4,
                            const float4* __restrict__ vel4, const float4* __restrict__ dacc,
                            const unsigned int* __restrict__ dcnt, const float4* __restrict__ ghost4,
                            const float4* __restrict__ facc, const float* __restrict__ fvsig,
                            const unsigned int* __restrict__ fcnt, const float* __restrict__ h, float gamma_gas,
                            void* out) {
  pdl_wait();
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
    const long long p = off + q;
    const long long i = (long long)perm[p] - off;
    const float H = Hs[p];
    const float ih = 1.0f / H;
    const float K3 = SPH_KNORM * ih * ih * ih;
    const float4 a = dacc[p];
    const float m = cen4[p].w;
    float* fo = reinterpret_cast<float*>(out);
    switch (field) {
      case SPH_FIELD_RHO: fo[i] = K3 * (a.x + m); break;
      case SPH_FIELD_DRHO_DH: fo[i] = -K3 * fmaf(3.0f, a.x + m, a.y) / h[perm[p]]; break;
      case SPH_FIELD_NW: fo[i] = K3 * (a.z + 1.0f); break;
      case SPH_FIELD_NNGB: fo[i] = (32.0f / 3.0f) * (a.z + 1.0f); break;
      case SPH_FIELD_COUNT: reinterpret_cast<int*>(out)[i] = (int)dcnt[p]; break;
      case SPH_FIELD_P: fo[i] = (gamma_gas - 1.0f) * ghost4[p].x * vel4[p].w; break;
      case SPH_FIELD_C: fo[i] = ghost4[p].z; break;
      case SPH_FIELD_F: fo[i] = a.y < 0.0f ? -3.0f * (a.x + m) / a.y : 1.0f; break;   // as the ghost pass
      case SPH_FIELD_A: {
        const float4 f = facc[p];
        fo[3 * i] = f.x;
        fo[3 * i + 1] = f.y;
        fo[3 * i + 2] = f.z;
        break;
      }
      case SPH_FIELD_DUDT: fo[i] = facc[p].w; break;
      case SPH_FIELD_VSIG: fo[i] = fvsig[p]; break;
      case SPH_FIELD_FORCE_COUNT: reinterpret_cast<int*>(out)[i] = (int)fcnt[p]; break;
      default: break;
    }
  }
}

// =========================================================================== launchers
// CTAs of a kernel resident per SM at SPH_THREADS threads (looked up once; engines
// may run in several host threads)
static int resident_ctas(const void* fn) {
  static std::mutex mu;
  static const void* fns[24] = {nullptr};   // the 12 density, 2 gathered density and 2 force instances
  static int val[24] = {0};
  std::lock_guard<std::mutex> lock(mu);
  for (int k = 0; k < 24; ++k) {
    if (fns[k] == fn) return val[k];
    if (!fns[k]) {
      int nb = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, SPH_THREADS, 0) != cudaSuccess || nb < 1) nb = 4;
      fns[k] = fn;
      val[k] = nb;
      return nb;
    }
  }
  return 4;
}

void launch_live_tasks(Engine& E, bool dens, const int* it_dev) {
  cudaMemsetAsync(E.Lq.n_live, 0, sizeof(unsigned int), E.st);
  // a captured rebuild step sizes the launch by the task capacity and the kernel
  // reads the counts of the build from the device
  const int cap_p = (int)E.l_ptask.n, cap_s = (int)E.l_stask.n;
  const long long npt = E.gcap ? -1 : E.n_ptasks, nst = E.gcap ? -1 : E.n_stasks;
  const long long n = E.gcap ? (long long)cap_p + cap_s : E.n_ptasks + E.n_stasks;
  if (n == 0) return;
  const int grid = (int)std::min<long long>((n + 255) / 256, (long long)E.nsm * 16);
  if (dens)
    launch_pdl(k_live_tasks<true>, grid, 256, E.st, E.Lq, E.T, E.TL, E.box.p, npt, nst, E.partial_pass, it_dev,
               cap_p, cap_s, it_dev ? E.gflag.p : nullptr, E.g_n.p, (unsigned int)E.g_live.n);
  else
    launch_pdl(k_live_tasks<false>, grid, 256, E.st, E.Lq, E.T, E.TL, E.box.p, npt, nst, 0, nullptr, cap_p, cap_s,
               nullptr, nullptr, 0u);
  count_launch();
}

// One density pass.  The kernel instance (first pass or later pass) follows the
// iteration counter it_dev when given, else E.partial_pass.  only: the instance
// the caller knows the pass needs (-1: both, as in a captured step, where the
// one that does not match the counter returns at once).
void launch_density(Engine& E, const int* it_dev, int only) {
  cudaMemsetAsync(E.task_ctr.p + 0, 0, sizeof(unsigned int), E.st);
  for (int part = 0; part < 2; ++part) {
    if (!it_dev && part != (E.partial_pass ? 1 : 0)) continue;
    if (it_dev && only >= 0 && part != only) continue;
    // compensated sums when asked, or (compensated < 0) from 100 neighbours on
    const bool kahan = E.prm.compensated > 0 || (E.prm.compensated < 0 && E.prm.n_ngb >= 100.0f);
    // the first pass records its pairs for the force pass when the records are on
    const bool rec = part == 0 && E.rec_valid;
    decltype(&k_density<false, false, false, false>) k;
    if (kahan)
      k = E.count_pairs ? (part ? k_density<true, true, true, false>
                                : (rec ? k_density<true, false, true, true> : k_density<true, false, true, false>))
                        : (part ? k_density<false, true, true, false>
                                : (rec ? k_density<false, false, true, true> : k_density<false, false, true, false>));
    else
      k = E.count_pairs ? (part ? k_density<true, true, false, false>
                                : (rec ? k_density<true, false, false, true> : k_density<true, false, false, false>))
                        : (part ? k_density<false, true, false, false>
                                : (rec ? k_density<false, false, false, true> : k_density<false, false, false, false>));
    launch_pdl(k, E.nsm * resident_ctas((const void*)k), SPH_THREADS, E.st,
        E.Lq, E.T, E.TL, E.box.p, E.pos4.p, E.cen4.p, E.sort_r.p, E.sort_i.p, E.act.p, E.perm.p, E.x.p, E.dacc.p,
        E.dcnt.p, E.pc.p, E.task_ctr.p + 0, E.partial_pass, it_dev, it_dev ? E.gflag.p : nullptr, E.g_n.p,
        (unsigned int)E.g_live.n, E.rec_for_force());
    count_launch();
  }
}

// The packing and the task list of a gathered later pass (a pass of the h
// iteration given by it_dev; the kernels decide on the device whether it gathers).
void launch_gather_prep(Engine& E, const int* it_dev) {
  // a captured rebuild step covers the capacities (this build's sizes are on the device)
  const long long nt = E.gcap ? E.N : E.n_tiles;
  const unsigned int* ntd = E.gcap ? reinterpret_cast<const unsigned int*>(E.dev_counters.p + 4) : nullptr;
  launch_pdl(k_pack_count, E.grid(32 * (nt + 1)), 256, E.st, nt, ntd, it_dev, E.TL, E.act.p, E.pk_cnt.p, E.g_n.p);
  count_launch();
  exclusive_scan(E.pk_cnt.p, E.pk_cnt.p, nt + 1, E.pk_sums.p, E.pk_tot.p + 0, E.st, ntd, it_dev);
  launch_pdl(k_pack_leaf, E.grid(nt + 1), 256, E.st, nt, ntd, it_dev, E.T, E.TL, E.pk_cnt.p, E.pk_v.p);
  count_launch();
  exclusive_scan(E.pk_v.p, E.pk_v.p, nt + 1, E.pk_sums.p, E.pk_tot.p + 1, E.st, ntd, it_dev);
  launch_pdl(k_pack_fill, E.grid(32 * nt), 256, E.st, nt, ntd, it_dev, E.T, E.TL, E.act.p, E.pk_cnt.p,
             E.pk_v.p, E.pk_idx.p, E.pk_info.p, E.pk_n.p);
  count_launch();
  const long long npair = E.gcap ? -1 : E.n_pairs, nself = E.gcap ? -1 : E.n_selfs;
  const long long nitem = E.gcap ? (long long)E.cap_pair + E.cap_self : (long long)E.n_pairs + E.n_selfs;
  const int allow = E.prm.h_gather != 0 && !E.count_pairs ? 1 : 0;
  launch_pdl(k_gather_tasks, E.grid(std::max<long long>(nitem, 1)), 256, E.st, E.Lq, E.T, npair, nself,
             E.cap_pair, E.cap_self, it_dev, (long long)E.N, allow, E.pk_v.p, E.pk_tot.p, E.g_live.p, E.g_n.p,
             (unsigned int)E.g_live.n, E.gflag.p);
  count_launch();
}

// The gathered density pass; returns at once unless the pass gathers.
void launch_density_gather(Engine& E) {
  const bool kahan = E.prm.compensated > 0 || (E.prm.compensated < 0 && E.prm.n_ngb >= 100.0f);
  const auto k = kahan ? k_density_gather<true> : k_density_gather<false>;
  cudaMemsetAsync(E.task_ctr.p + 2, 0, sizeof(unsigned int), E.st);
  launch_pdl(k, E.nsm * resident_ctas((const void*)k), SPH_THREADS, E.st, E.Lq, E.T, E.TL, E.box.p, E.pos4.p,
             E.cen4.p, E.perm.p, E.x.p, E.dacc.p, E.dcnt.p, E.g_live.p, E.g_n.p, (unsigned int)E.g_live.n,
             E.gflag.p, E.pk_info.p, E.pk_n.p, E.pk_idx.p, E.task_ctr.p + 2);
  count_launch();
}

#ifndef FORCE_BLOCKS
#define FORCE_BLOCKS 0
#endif
void launch_force(Engine& E) {
  const auto k = E.count_pairs ? k_force<true> : k_force<false>;
  cudaMemsetAsync(E.task_ctr.p + 1, 0, sizeof(unsigned int), E.st);
  int nb = resident_ctas((const void*)k);
  if (FORCE_BLOCKS > 0) {
    static bool set[2] = {false, false};
    if (!set[E.count_pairs ? 1 : 0]) {
      const int pct = (int)std::ceil(100.0 * FORCE_BLOCKS * (sizeof(ForceShared) * SPH_WARPS_PER_CTA + 1024) / (228.0 * 1024));
      cudaFuncSetAttribute((const void*)k, cudaFuncAttributePreferredSharedMemoryCarveout, std::min(pct, 100));
      set[E.count_pairs ? 1 : 0] = true;
    }
    nb = std::min(nb, FORCE_BLOCKS);
  }
  launch_pdl(k, E.nsm * nb, SPH_THREADS, E.st,
      E.Lq, E.T, E.TL, E.box.p, E.pos4.p, E.cen4.p, E.vel4.p, E.ghost4.p, E.sort_r.p, E.sort_i.p, E.perm.p, E.x.p,
      E.prm.alpha_visc, E.facc.p, E.fvsig.p, E.fcnt.p, E.pc.p, E.task_ctr.p + 1, E.rec_for_force());
  count_launch();
}

void launch_ghost(Engine& E, int mode, int it, const int* it_dev) {
  launch_pdl(k_ghost, E.grid(E.N), 256, E.st, E.N, mode, it, it_dev, E.prm.h_max_iter, E.prm.gamma_kernel, E.prm.n_ngb,
                                          E.prm.h_tol, E.prm.gamma_gas, E.perm.p, E.Hs.p, E.pos4.p, E.cen4.p,
                                          E.vel4.p, E.dacc.p, E.act.p, E.h.p, E.hlo.p, E.hhi.p, E.conv.p,
                                          E.hlimp.p, E.leaf_of.p, E.T, E.ghost4.p, E.hhist.p, E.dev_counters.p,
                                          E.err_all.p); count_launch();
}

void launch_zero_density(Engine& E, bool all) {
  launch_pdl(k_zero_active, E.grid(E.N), 256, E.st, E.N, E.act.p, E.dacc.p, E.dcnt.p, all ? 1 : 0); count_launch();
}

void launch_set_active(Engine& E) {
  E.partial_pass = 0;
  launch_pdl(k_set_active, E.grid(E.N), 256, E.st, E.N, E.act.p); count_launch();
  cudaMemsetAsync(E.t_active.p, 1, E.gcap ? (size_t)E.cap_nodes : (size_t)E.n_nodes, E.st);
  cudaMemsetAsync(E.tl_active.p, 1, E.gcap ? (size_t)E.N : (size_t)E.n_tiles, E.st);
}

void launch_count_unconverged(Engine& E, int* out) {
  launch_pdl(k_count_unconverged, E.grid(E.N), 256, E.st, E.N, E.conv.p, out); count_launch();
}

void launch_mark_active_cells(Engine& E) {
  E.partial_pass = 1;
  // a captured rebuild step covers the capacities (this build's sizes are on the device)
  const long long nn = E.gcap ? E.cap_nodes : E.n_nodes, nt = E.gcap ? E.N : E.n_tiles;
  cudaMemsetAsync(E.t_active.p, 0, nn, E.st);
  cudaMemsetAsync(E.tl_active.p, 0, nt, E.st);
  cudaMemsetAsync(E.t_alo.p, 0xff, 3 * (size_t)nn * sizeof(unsigned int), E.st);
  cudaMemsetAsync(E.t_ahi.p, 0, 3 * (size_t)nn * sizeof(unsigned int), E.st);
  launch_pdl(k_mark_active, E.grid(32 * nt), 256, E.st, nt,
             E.gcap ? reinterpret_cast<const unsigned int*>(E.dev_counters.p + 4) : nullptr, E.act.p, E.pos4.p, E.T,
             E.TL);
  count_launch();
}

void launch_task_offsets(Engine& E) {
  launch_pdl(k_task_tiles, E.grid(E.cap_pair + E.cap_self), 256, E.st, E.Lq, E.T, E.cap_pair, E.cap_self); count_launch();
  exclusive_scan(E.Lq.p_toff, E.Lq.p_toff, E.cap_pair, E.scan_tmp.p,
                 reinterpret_cast<unsigned int*>(E.Lq.counts + 6), E.st);
  exclusive_scan(E.Lq.s_toff, E.Lq.s_toff, E.cap_self, E.scan_tmp.p,
                 reinterpret_cast<unsigned int*>(E.Lq.counts + 7), E.st);
}

void launch_task_items(Engine& E) {
  launch_pdl(k_task_items, E.nsm * 8, 256, E.st, E.Lq, E.T, E.gcap ? -1 : E.n_pairs, E.gcap ? -1 : E.n_selfs,
             E.cap_pair, E.cap_self, (unsigned int)E.l_ptask.n, (unsigned int)E.l_stask.n);
  count_launch();
}

void launch_bracket_reset(Engine& E) {
  launch_pdl(k_h_bracket_reset, E.grid(E.N), 256, E.st, E.N, E.hlo.p, E.hhi.p, E.conv.p); count_launch();
}

void launch_reduce(Engine& E) {
  cudaMemsetAsync(E.red.p, 0, sizeof(double) * 8 * E.nbox, E.st);
  long long maxn = 1;
  for (int b = 0; b < E.nbox; ++b) maxn = std::max(maxn, E.spec[b].n);
  const int gx = (int)std::max<long long>(1, std::min<long long>((maxn + 255) / 256, (E.nsm * 4 + E.nbox - 1) / E.nbox));
  launch_pdl(k_reduce, dim3(gx, std::min(E.nbox, 65535)), 256, E.st, E.nbox, E.boff.p, E.box.p, E.perm.p, E.cen4.p,
             E.vel4.p, E.facc.p,
                                                                 E.red.p); count_launch();
}

cudaError_t add_cond_set_node(cudaGraphNode_t* node, cudaGraph_t g, const cudaGraphNode_t* deps, size_t ndeps,
                              cudaGraphConditionalHandle h, const int* flag) {
  cudaKernelNodeParams kp = {};
  void* args[2] = {&h, &flag};
  kp.func = (void*)k_cond_set;
  kp.gridDim = dim3(1);
  kp.blockDim = dim3(1);
  kp.sharedMemBytes = 0;
  kp.kernelParams = args;
  kp.extra = nullptr;
  return cudaGraphAddKernelNode(node, g, deps, ndeps, &kp);
}

void launch_cond_keep(Engine& E, cudaGraphConditionalHandle keep) {
  launch_pdl(k_cond_keep, 1, 1, E.st, keep, E.reuse_flag.p); count_launch();
}

void launch_iter_start(Engine& E, cudaGraphConditionalHandle iter) {
  launch_pdl(k_iter_start, 1, 1, E.st, iter, E.it_dev.p); count_launch();
}

void launch_iter_step(Engine& E) {
  launch_pdl(k_iter_step, 1, 1, E.st, E.it_dev.p, E.dev_counters.p, E.err_all.p, E.prm.h_max_iter); count_launch();
}

void launch_iter_next(Engine& E, cudaGraphConditionalHandle iter, cudaGraphConditionalHandle force) {
  launch_pdl(k_iter_next, 1, 1, E.st, iter, force, E.it_dev.p, E.dev_counters.p, E.err_all.p, E.prm.h_max_iter,
                                 E.it_dev.p + 1); count_launch();
}

void launch_set_drift(Engine& E) {
  launch_pdl(k_set_drift, 1, 256, E.st, E.nbox, E.box.p, E.dmax_bits.p); count_launch();
}

void launch_save_acc(Engine& E) { launch_pdl(k_save_acc, E.grid(E.N), 256, E.st, E.N, E.perm.p, E.facc.p, E.a_in.p); count_launch(); }

void launch_kick(Engine& E) { launch_pdl(k_kick, E.grid(E.N), 256, E.st, E.N, E.bid.p, E.box.p, E.a_in.p, E.v.p, E.u.p); count_launch(); }

// one more root kept by every moving box (the ghost pass of the step writes it)
__global__ void k_hlev_next(int nbox, const BoxDesc* __restrict__ box, int* __restrict__ hlev) {
  pdl_wait();
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nbox; b += gridDim.x * blockDim.x)
    if (box[b].dt != 0.0) hlev[b] = min(hlev[b] + 1, 3);
}

// history levels of the boxes of a new layout: a moved box keeps its own
__global__ void k_remap_hlev(int nbox, const long long* __restrict__ src_tab, const int* __restrict__ old_lev,
                             int* __restrict__ lev) {
  pdl_wait();
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nbox; b += gridDim.x * blockDim.x) {
    const long long s = src_tab[b];
    lev[b] = s >= 0 ? old_lev[s] : 0;
  }
}

// h of one box set from src (device); the box's root history restarts when any h changes
__global__ void k_set_h(long long n, const float* __restrict__ src, float* __restrict__ h, int* __restrict__ hlev) {
  pdl_wait();
  bool diff = false;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float s = src[i];
    diff |= __float_as_uint(s) != __float_as_uint(h[i]);
    h[i] = s;
  }
  if (__syncthreads_or(diff) && threadIdx.x == 0) *hlev = 0;
}

void launch_drift(Engine& E) {
  launch_pdl(k_drift, E.grid(E.N), 256, E.st, E.N, E.bid.p, E.box.p, E.x.p, E.v.p, E.h.p, E.hhist.p, E.hlev.p);
  count_launch();
  launch_pdl(k_hlev_next, 1, 256, E.st, E.nbox, E.box.p, E.hlev.p); count_launch();
}

void launch_set_h(Engine& E, int b, const float* src) {
  const long long n = E.spec[b].n;
  if (n == 0) return;
  launch_pdl(k_set_h, E.grid(n), 256, E.st, n, src, E.h.p + E.off[b], E.hlev.p + b); count_launch();
}

void launch_get_field(Engine& E, long long off, long long n, int field, void* out) {
  launch_pdl(k_get_field, E.grid(n), 256, E.st, off, n, field, E.perm.p, E.Hs.p, E.cen4.p, E.vel4.p, E.dacc.p, E.dcnt.p,
                                           E.ghost4.p, E.facc.p, E.fvsig.p, E.fcnt.p, E.h.p, E.prm.gamma_gas, out);
  count_launch();
}

}  // namespace sph
