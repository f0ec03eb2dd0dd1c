// Density pass that allocates nothing, for callers that cannot call cudaMalloc.
//
// Some callers run where device allocation is not allowed: inside an
// allocator-free embedding (a pre-sized arena owned by someone else), from code
// that must not trigger the driver's allocator after start-up, or where every
// allocation has to be accounted for up front.  sph_density_static serves them:
// it takes device pointers for its inputs and outputs and keeps all of its
// working memory in one fixed device array that exists from the moment the
// library is loaded, so no call allocates.
//
// The working memory is the static array below: a uniform cell list of the
// box (cell counts, offsets, fill cursors) and the particle indices sorted by
// cell.  One thread block builds it and then evaluates, for every particle,
// rho_i = sum_{r_ij < H_i} m_j W(r_ij, H_i) (j = i included) and the neighbour
// count, with the neighbour decision r_ij < H taken in FP64 in the same fixed
// evaluation order as the main path's exact decision, so counts match it
// bit for bit.
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>

#include "sph.h"
#include "sph_internal.cuh"

namespace {

constexpr int kMaxN = SPH_STATIC_MAX_N;           // particles per call
constexpr int kMaxSide = 32;                      // cells per dimension of the cell list
constexpr int kMaxCells = kMaxSide * kMaxSide * kMaxSide;
constexpr int kThreads = 1024;

// Layout of the static working memory (all 4-byte words):
//   [0, kMaxCells)                 cell counts, then exclusive offsets
//   [kMaxCells, 2 kMaxCells)       fill cursors
//   [2 kMaxCells, 2 kMaxCells + kMaxN)   particle indices sorted by cell
//   [.. + kMaxN]                   support radius H of every particle (FP32 bits)
constexpr size_t kScratchWords = 2 * (size_t)kMaxCells + 2 * (size_t)kMaxN + 64;

// The working memory: held by every device that loads the library, for the
// life of the process.  Host code must not use this name as a device address.
static __device__ __align__(256) unsigned int g_scratch[kScratchWords];

// Device address of g_scratch per device, looked up once per device.  Host
// threads that make their first calls at the same time may each look it up; they
// store the same value, through atomics.
static std::atomic<unsigned int*> g_scratch_ptr[64];

__device__ __forceinline__ int wrap_cell(int c, int side, int periodic) {
  if (periodic) return (c + side) % side;
  return c;
}

__global__ void __launch_bounds__(kThreads) k_density_static(const double* __restrict__ x,
                                                            const float* __restrict__ m,
                                                            const float* __restrict__ h, int n, double L,
                                                            int periodic, float gamma_k, float* __restrict__ rho,
                                                            int* __restrict__ count, unsigned int* __restrict__ ws,
                                                            int* __restrict__ status) {
  __shared__ float s_hmax;
  __shared__ int s_bad;
  __shared__ int s_side;
  __shared__ unsigned int s_carry;
  unsigned int* cells = ws;
  unsigned int* cursor = ws + kMaxCells;
  unsigned int* order = ws + 2 * kMaxCells;
  float* Hs = reinterpret_cast<float*>(ws + 2 * kMaxCells + kMaxN);
  const int tid = threadIdx.x;
  if (tid == 0) {
    s_hmax = 0.0f;
    s_bad = 0;
    *status = 0;
  }
  __syncthreads();
  // input checks (those of the main path's ingest: 0 <= x < L, h and m finite and
  // positive), support radii and their maximum
  float hm = 0.0f;
  bool bad = false;
  for (int i = tid; i < n; i += kThreads) {
    const float hi = h[i], mi = m[i];
    for (int k = 0; k < 3; ++k) {
      const double xk = x[3 * i + k];
      bad |= !(xk >= 0.0 && xk < L);
    }
    bad |= !(isfinite(hi) && hi > 0.0f) || !(isfinite(mi) && mi > 0.0f);
    const float H = __fmul_rn(gamma_k, hi);
    Hs[i] = H;
    if (H > hm) hm = H;
  }
  hm = warp_max(hm);
  if ((tid & 31) == 0) atomic_max_pos(&s_hmax, hm);
  if (bad) s_bad = 1;
  __syncthreads();
  if (tid == 0) {
    // cells of edge >= H_max (with a relative margin far above the rounding of a
    // cell index); at least 3 per dimension for periodic boxes
    int side = 1;
    if (s_bad || !(s_hmax > 0.0f) || !isfinite(s_hmax)) {
      *status = SPH_E_INVALID;
    } else {
      const double sd = floor(L / ((double)s_hmax * (1.0 + 1e-9)));
      side = sd < 1.0 ? 1 : (sd > (double)kMaxSide ? kMaxSide : (int)sd);
      if (periodic && side < 3) *status = SPH_E_H_TOO_LARGE;
    }
    s_side = side;
  }
  __syncthreads();
  if (*status != 0) return;
  const int side = s_side;
  const int ncell = side * side * side;
  const double scale = (double)side / L;
  // the working memory keeps the previous call's contents: clear the counts
  for (int c = tid; c < ncell; c += kThreads) cells[c] = 0;
  __syncthreads();
  for (int i = tid; i < n; i += kThreads) {
    int c[3];
    for (int k = 0; k < 3; ++k) {
      int q = (int)floor(x[3 * i + k] * scale);
      c[k] = q < 0 ? 0 : (q >= side ? side - 1 : q);
    }
    atomicAdd(&cells[(c[2] * side + c[1]) * side + c[0]], 1u);
  }
  __syncthreads();
  // exclusive scan of the counts (one block, in chunks of kThreads)
  if (tid == 0) s_carry = 0;
  __syncthreads();
  __shared__ unsigned int s_tmp[kThreads / 32];
  for (int base = 0; base < ncell; base += kThreads) {
    const int c = base + tid;
    const unsigned int v = c < ncell ? cells[c] : 0u;
    unsigned int incl = v;
    const int lane = tid & 31, w = tid >> 5;
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) s_tmp[w] = incl;
    __syncthreads();
    if (w == 0) {
      unsigned int t = s_tmp[lane];
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned int y = __shfl_up_sync(0xffffffffu, t, o);
        if (lane >= o) t += y;
      }
      s_tmp[lane] = t;
    }
    __syncthreads();
    const unsigned int excl = s_carry + (w > 0 ? s_tmp[w - 1] : 0u) + incl - v;
    if (c < ncell) {
      cells[c] = excl;
      cursor[c] = excl;
    }
    __syncthreads();
    if (tid == 0) s_carry += s_tmp[31];
    __syncthreads();
  }
  for (int i = tid; i < n; i += kThreads) {
    int c[3];
    for (int k = 0; k < 3; ++k) {
      int q = (int)floor(x[3 * i + k] * scale);
      c[k] = q < 0 ? 0 : (q >= side ? side - 1 : q);
    }
    order[atomicAdd(&cursor[(c[2] * side + c[1]) * side + c[0]], 1u)] = (unsigned int)i;
  }
  __syncthreads();
  // density of every particle over the neighbouring cells
  const double halfL = 0.5 * L;
  for (int i = tid; i < n; i += kThreads) {
    const double xi[3] = {x[3 * i], x[3 * i + 1], x[3 * i + 2]};
    const float Hi = Hs[i];
    const float invH = 1.0f / Hi;
    int ci[3];
    for (int k = 0; k < 3; ++k) {
      int q = (int)floor(xi[k] * scale);
      ci[k] = q < 0 ? 0 : (q >= side ? side - 1 : q);
    }
    float sw = 0.0f;
    int cnt = 0;
    for (int dz = -1; dz <= 1; ++dz)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          const int cx = wrap_cell(ci[0] + dx, side, periodic), cy = wrap_cell(ci[1] + dy, side, periodic),
                    cz = wrap_cell(ci[2] + dz, side, periodic);
          if (cx < 0 || cy < 0 || cz < 0 || cx >= side || cy >= side || cz >= side) continue;
          const int c = (cz * side + cy) * side + cx;
          const unsigned int e = (c + 1 < ncell) ? cells[c + 1] : (unsigned int)n;
          for (unsigned int q = cells[c]; q < e; ++q) {
            const unsigned int j = order[q];
            if ((int)j == i) continue;
            const double xj[3] = {x[3 * j], x[3 * j + 1], x[3 * j + 2]};
            const double r2 = canonical_r2(xi, xj, L, halfL, periodic);
            if (!canonical_less(r2, Hi)) continue;
            float w, dw;
            spline_w_dw((float)sqrt(r2) * invH, w, dw);
            sw = fmaf(m[j], w, sw);
            ++cnt;
          }
        }
    const float K3 = SPH_KNORM * invH * invH * invH;
    rho[i] = K3 * (sw + m[i]);
    count[i] = cnt;
  }
}

}  // namespace

extern "C" sph_status sph_density_static(const double* x, const float* m, const float* h, int64_t n, double box_len,
                                         int periodic, float* rho, int32_t* count, void* stream) {
  if (!x || !m || !h || !rho || !count || !(box_len > 0)) return SPH_E_INVALID;
  if (n < 1 || n > kMaxN) return SPH_E_INVALID;      // beyond the static working memory
  if (!std::isfinite(box_len)) return SPH_E_INVALID;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return SPH_E_CUDA;
  unsigned int* ws = g_scratch_ptr[dev].load(std::memory_order_acquire);
  if (!ws) {
    // first call on this device: look up the array's device address (call it
    // before any stream capture)
    unsigned int* ptr = nullptr;
    if (cudaGetSymbolAddress(reinterpret_cast<void**>(&ptr), g_scratch) != cudaSuccess || !ptr) return SPH_E_CUDA;
    g_scratch_ptr[dev].store(ptr, std::memory_order_release);
    ws = ptr;
  }
  // the status word lives in the last words of the working memory
  int* status = reinterpret_cast<int*>(ws + kScratchWords - 1);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  k_density_static<<<1, kThreads, 0, st>>>(x, m, h, (int)n, box_len, periodic ? 1 : 0, SPH_STATIC_GAMMA_K, rho,
                                            count, ws, status);
  if (cudaGetLastError() != cudaSuccess) return SPH_E_CUDA;
  int hs = 0;
  if (cudaMemcpyAsync(&hs, status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess) return SPH_E_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return SPH_E_CUDA;
  return hs == 0 ? SPH_OK : (sph_status)hs;
}
