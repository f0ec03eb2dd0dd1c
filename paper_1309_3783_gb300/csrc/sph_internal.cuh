// Internal definitions of the GB300 SPH path: device data layout and helpers
// shared by the build, interaction and host translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <utility>

// Programmatic dependent launch.  The library's kernels are launched with
// programmatic stream serialisation (launch_pdl), so that a kernel's launch
// overlaps the end of the kernel before it in the stream instead of starting
// after it.  Every kernel begins with pdl_wait(), which blocks until the
// previous grid has completed and its memory writes are visible: each kernel
// still sees all the work issued before it, as in plain stream order.  No
// kernel signals its dependents early.  While the stream is being captured into
// a graph the launches are plain (the captured step keeps ordinary edges).
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, cudaStream_t st, Args&&... args) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  const cudaError_t e = cudaStreamIsCapturing(st, &cs);
  if (e != cudaSuccess) return e;
  if (cs != cudaStreamCaptureStatusNone) {
    kernel<<<grid, block, 0, st>>>(std::forward<Args>(args)...);
    return cudaGetLastError();
  }
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

#define SPH_MAX_DEPTH 20          // bits per dimension of the Morton code
#define SPH_WARPS_PER_CTA 4
#define SPH_THREADS (32 * SPH_WARPS_PER_CTA)
#define SORT_SMALL 2048u       // cells with up to this many clusters are sorted in shared memory
#define SORT_NONE 0xffffffffu  // sortbase of a cell whose clusters are not sorted

// Error bits set by kernels in a box's status word.
enum : unsigned int {
  ERR_BAD_INPUT = 1u,        // NaN / non-positive h / x outside [0, L)
  ERR_H_TOO_LARGE = 2u,      // top grid cannot hold H_max
  ERR_OVERFLOW = 4u,         // a device list exceeded its capacity
  ERR_REBUILD = 8u,          // some H outgrew what the cell splits assumed
  ERR_DEPTH = 16u,           // a split was blocked by a depth bound below the full depth
  ERR_SHAPE = 32u,           // a captured build's top levels no longer fit the boxes' support radii
};

// One box of a batch.  Particles of box b occupy [off, off + n) both in the
// caller-order input arrays and in the key-sorted arrays.
struct BoxDesc {
  double L, invL;       // edge and its reciprocal
  double margin;        // 2^-50 L: every cell rule is strict by this much
  long long off, n;
  int periodic;
  int k;                // top level: cell edge L / 2^k
  float Hmax, Hmin;     // extremes of the support radius (physical units)
  unsigned int err;     // ERR_* bits
  unsigned int pow2;    // 1 when L is a power of two: x / L is then exactly x * invL
  float drift2;         // twice the largest displacement since the decomposition was built (physical)
  float drift_u;        // the largest displacement since the build (units of L)
  double dt;            // time step of the box (0: passes only)
  double dt_prev[3];    // time steps of the box's three previous steps
  float hw[4][4];       // extrapolation weights of the last roots at the new time, row l for
                        //   l earlier roots besides the last (the box's level, kept on the device)
  long long nown;         // the box's first nown particles (caller order) enter the conservation
                          //   sums; the others are a halo of particles owned elsewhere
  unsigned int global32;  // 1: plain FP32 positions (x / L rounded to FP32 in the box frame; the
                          //   offsets are taken from them); 0: offsets from the FP64 positions
};

// The 13 cell-pair directions db in {-1,0,1}^3 with dz > 0, or dz = 0 and
// dy > 0, or dz = dy = 0 and dx > 0 (one of each +-db).  Section II-C: the
// sorted indices are kept per cell along these 13 axes.
__host__ __device__ inline void axis_vec(int a, int& dx, int& dy, int& dz) {
  // enumeration in z-major order over (dx, dy, dz) restricted to the half space:
  // 0: (1, 0, 0); 1..3: (a - 2, 1, 0); 4..12: ((a - 4) % 3 - 1, (a - 4) / 3 - 1, 1).
  // Computed, not looked up: a table indexed at run time would be built in local
  // memory at every call.
  if (a == 0) {
    dx = 1; dy = 0; dz = 0;
  } else if (a < 4) {
    dx = a - 2; dy = 1; dz = 0;
  } else {
    const int b = a - 4;
    dx = b % 3 - 1; dy = b / 3 - 1; dz = 1;
  }
}

__host__ __device__ inline int axis_index(int dx, int dy, int dz) {
  // inverse of axis_vec for db in the positive half space; -1 otherwise
  if (dz == 1) return 4 + (dy + 1) * 3 + (dx + 1);
  if (dz == 0 && dy == 1) return 1 + (dx + 1);
  if (dz == 0 && dy == 0 && dx == 1) return 0;
  return -1;
}

__host__ __device__ inline bool dir_positive(int dx, int dy, int dz) {
  return dz > 0 || (dz == 0 && (dy > 0 || (dy == 0 && dx > 0)));
}

// ---------------------------------------------------------------- Morton codes
__host__ __device__ inline unsigned long long spread3(unsigned long long v) {
  v &= 0x1fffffull;
  v = (v | (v << 32)) & 0x1f00000000ffffull;
  v = (v | (v << 16)) & 0x1f0000ff0000ffull;
  v = (v | (v << 8)) & 0x100f00f00f00f00full;
  v = (v | (v << 4)) & 0x10c30c30c30c30c3ull;
  v = (v | (v << 2)) & 0x1249249249249249ull;
  return v;
}

__host__ __device__ inline unsigned int compact3(unsigned long long v) {
  v &= 0x1249249249249249ull;
  v = (v ^ (v >> 2)) & 0x10c30c30c30c30c3ull;
  v = (v ^ (v >> 4)) & 0x100f00f00f00f00full;
  v = (v ^ (v >> 8)) & 0x1f0000ff0000ffull;
  v = (v ^ (v >> 16)) & 0x1f00000000ffffull;
  v = (v ^ (v >> 32)) & 0x1fffffull;
  return (unsigned int)v;
}

// x in bits 0,3,6..., y in 1,4,..., z in 2,5,...
__host__ __device__ inline unsigned long long morton3(unsigned int x, unsigned int y, unsigned int z) {
  return spread3(x) | (spread3(y) << 1) | (spread3(z) << 2);
}

// ------------------------------------------------------------ cubic spline
// w(q) and dw/dq of the cubic spline with support 1 (W = 8/(pi H^3) w(r/H)).
__device__ __forceinline__ void spline_w_dw(float q, float& w, float& dw) {
  const float one_m = 1.0f - q;
  const float q2 = q * q;
  const float w_in = fmaf(6.0f * q2, q - 1.0f, 1.0f);      // 1 - 6q^2 + 6q^3
  const float dw_in = q * fmaf(18.0f, q, -12.0f);          // -12q + 18q^2
  const float w_out = 2.0f * one_m * one_m * one_m;        // 2(1-q)^3
  const float dw_out = -6.0f * one_m * one_m;              // -6(1-q)^2
  const bool inner = q < 0.5f;
  w = inner ? w_in : w_out;
  dw = inner ? dw_in : dw_out;
}

#define SPH_KNORM 2.5464790894703255f   // 8 / pi

// ------------------------------------------------- orderable float as uint32
__device__ __forceinline__ unsigned int float_key(float f) {
  unsigned int u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float key_float(unsigned int k) {
  return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

// ------------------------------------------- exact neighbour decision in FP64
// The fixed evaluation both this path and the oracle use for r_ij < H:
// d = x_i - x_j per component, wrapped by +-L when |d| > L/2 (periodic),
// r2 = (d0*d0 + d1*d1) + d2*d2 with correctly rounded operations, no FMA.
__device__ __forceinline__ double canonical_r2(const double* xi, const double* xj, double L, double halfL,
                                               int periodic) {
  double d[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    double t = __dsub_rn(xi[k], xj[k]);
    if (periodic) {
      if (t > halfL) t = __dsub_rn(t, L);
      else if (t < -halfL) t = __dadd_rn(t, L);
    }
    d[k] = t;
  }
  return __dadd_rn(__dadd_rn(__dmul_rn(d[0], d[0]), __dmul_rn(d[1], d[1])), __dmul_rn(d[2], d[2]));
}

__device__ __forceinline__ bool canonical_less(double r2, float H) {
  const double h = (double)H;
  return r2 < __dmul_rn(h, h);   // exact: the product of two FP32 fits FP64
}

// ------------------------------------------------------------ warp helpers
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ float warp_min(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// atomicMax / atomicMin on non-negative floats and doubles through their bits
__device__ __forceinline__ void atomic_max_pos(float* a, float v) {
  atomicMax(reinterpret_cast<unsigned int*>(a), __float_as_uint(v));
}
__device__ __forceinline__ void atomic_min_pos(float* a, float v) {
  atomicMin(reinterpret_cast<unsigned int*>(a), __float_as_uint(v));
}
__device__ __forceinline__ void atomic_min_pos(double* a, double v) {
  atomicMin(reinterpret_cast<unsigned long long*>(a), (unsigned long long)__double_as_longlong(v));
}

// ------------------------------------------------------------ device arrays
// Cell tree (structure of arrays, capacity cap_nodes).
struct Tree {
  unsigned int* start;      // first particle (sorted order)
  unsigned int* count;
  unsigned long long* key;  // box bits | Morton prefix of the cell at its level
  int* level;
  int* box;
  int* child;               // first child (children are contiguous), -1 for a leaf
  int* nchild;
  int* parent;
  int* split;               // 1 when split
  float* hmax;              // max support radius inside (physical units); grows with H
  unsigned int* nsmall;     // particles with H < edge/2 - margin
  double* hlim;             // H must stay below this for the interactions built (physical)
  float4* cen;              // centre minus its top cell's centre (units of L), exact
  unsigned int* axes;       // bit a: a sorted list along axis a is needed
  unsigned int* sortbase;   // offset of the first sorted list of this cell
  unsigned char* active;    // 1 when a particle inside still iterates h
  unsigned char* changed;   // 1 when a particle inside took a new h after the first density pass
  unsigned int* clo;        // box of those particles, relative to the cell centre (units of L),
  unsigned int* chi;        //   3 orderable float keys each
  unsigned int* alo;        // box of the particles still iterating h, relative to the
  unsigned int* ahi;        //   cell centre (units of L), 3 orderable float keys each
  unsigned int* tile0;      // first cluster of the cell (clusters of a cell are contiguous)
  unsigned int* ntile;      // clusters of the cell
  int* n_nodes;             // [0] nodes in use, [1] first node of the frontier, [2] end of frontier,
                            // [3] top cells, [4] blocks done with the current tree round,
                            // [5] deepest level holding a cell
};

// Clusters: runs of at most 32 (the cluster size) consecutive particles of one leaf (particles of a
// leaf are ordered by H class, then Morton order), the unit the interaction
// kernels load into a warp.  Their boxes and largest H drive the culling.
struct Tiles {
  unsigned int* start;      // first particle (sorted order)
  unsigned int* n;          // particles in the cluster (1..32)
  unsigned int* leaf;       // leaf cell
  float4* lo;               // box minimum relative to the leaf centre (units of L); w: max H (physical)
  float4* hi;               // box maximum relative to the leaf centre (units of L)
  float4* cen;              // the leaf's centre (as Tree::cen)
  unsigned char* active;    // 1 when a particle inside still iterates h
  unsigned char* changed;   // 1 when a particle inside took a new h after the first density pass
};

// The interacting pairs of the first (full) density pass of an h iteration, kept
// for the force pass: per batch of staged partners, the partners' particle
// indices and, per particle of the warp's cluster, the mask of the partners it
// interacts with (r < max(H_i, H_j), decided exactly).  A warp appends its batches
// to chunks of REC_CHUNK batches that it takes from a counter and links; the
// batches of one task are consecutive in that chain.
constexpr unsigned int REC_CHUNK = 32;
constexpr unsigned int REC_NONE = 0xffffffffu;
struct PairRec {
  unsigned int* pool;       // 64 words per batch: 32 partner indices (REC_NONE: empty slot), 32 masks
  unsigned int* next;       // per chunk: the chunk its warp continued in
  unsigned int* ctr;        // [0] chunks taken (may run past cap: those batches are not kept)
  uint2* ptask;             // per pair task: (first batch, batches); x = REC_NONE: not recorded
  uint2* stask;             // per self task
  unsigned int cap;         // chunks in the pool
};

// Interaction lists.
struct Lists {
  int* self_a;              // final self-interactions
  int* pair_a;              // final pair-interactions: cells a, b, axis (a -> b)
  int* pair_b;
  int* pair_axis;
  int* q_kind[2];           // expansion queues (ping-pong): 0 self, 1 pair
  int* q_a[2];
  int* q_b[2];
  int* q_axis[2];
  unsigned int* p_toff;     // per pair: first task (i-tile) number, exclusive prefix
  unsigned int* s_toff;     // per self: first task number
  unsigned int* p_task;     // per pair task: its pair
  unsigned int* s_task;     // per self task: its self
  uint2* p_live;            // pair tasks of the current pass that have work: (pair, cluster)
  unsigned int* n_live;     // their number
  int* counts;              // [0] selfs, [1] pairs, [2] queue 0 size, [3] queue 1 size, [4] sort segments,
                            // [5] sort entries, [6] pair tasks, [7] self tasks
};

// Per-box counters kept by the pair kernels when counting is on.
struct PairCounters {
  unsigned long long dens_pairs, dens_sides, dens_cand, force_pairs, force_cand, rechecks;
};
