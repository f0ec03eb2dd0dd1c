// Host orchestration of the GB300 SPH path and the C-ABI of include/sph.h.
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "sph_engine.h"

namespace sph {

// kernels of build.cu
__global__ void k_ingest(long long, const int*, BoxDesc*, const double*, const float*, const float*, const float*,
                         const float*, float, float*);
__global__ void k_keys(long long, int, const int*, const BoxDesc*, const double*, unsigned long long*, unsigned int*);
__global__ void k_box_ids(long long, int, const long long*, int*);
__global__ void k_displacement(long long, const int*, const BoxDesc*, const double*, const double*,
                               unsigned long long*);
__global__ void k_reuse_limits(long long, int, const unsigned long long*, Tree, const unsigned int*,
                               const unsigned int*, const float*, float, const unsigned long long*, float*,
                               unsigned int*);
__global__ void k_leaf_hmax(Tree, int, const float*);
__global__ void k_tile_boxes(long long, Tiles, const float4*);
__global__ void k_relayout(const long long*, const double*, const float*, const float*, const float*, const float*,
                           const float4*, const float4*, double*, float*, float*, float*, float*, float4*, float4*);
__global__ void k_gather_sorted(long long, const unsigned int*, const float*, const float*, const float*, const int*,
                                const BoxDesc*, const float4*, int, float*, float4*);
__global__ void k_top_nodes(long long, int, int, const BoxDesc*, const unsigned long long*, Tree, int, int*,
                            unsigned int*);
__global__ void k_tree_round(Tree, const BoxDesc*, const float*, const unsigned long long*, int, int, float, int,
                             int, int, unsigned int*);
__global__ void k_frontier_init(Tree, int);
__global__ void k_items_top(int, Tree, const BoxDesc*, const unsigned long long*, const int*, int, int, Lists, int,
                            unsigned int*);
__global__ void k_items_expand(int, Tree, const BoxDesc*, Lists, int, int, int, unsigned int*, float);
__global__ void k_leaves(Tree, int, unsigned int*);
__global__ void k_particle_limits(long long, Tree, const unsigned int*, float*);
__global__ void k_shift(long long, int, const unsigned long long*, const unsigned int*, const unsigned int*, Tree,
                        const BoxDesc*, const double*, const float*, const float*, float4*, float4*);
__global__ void k_mark_axes(Lists, int, Tree);
__global__ void k_sort_alloc(Tree, int, Lists, int*, int*, unsigned int*, unsigned long long*, int, uint4*,
                             unsigned int*, unsigned int, unsigned int, unsigned int*);
__global__ void k_sort_small(const uint4*, const unsigned int*, Tree, Tiles, float*, unsigned int*);
__global__ void k_sort_merge(const uint4*, const unsigned int*, Tree, Tiles, float*, unsigned int*);
__global__ void k_sort_big_keys(int, const int*, const int*, const unsigned int*, Tree, Tiles, unsigned long long*,
                                unsigned int*, const unsigned long long*, int);
__global__ void k_sort_big_scatter(int, const int*, const int*, const unsigned int*, Tree, Tiles,
                                   const unsigned int*, float*, unsigned int*, const unsigned long long*, int);
__global__ void k_leaf_partition(Tree, int, const BoxDesc*, const float*, unsigned int*);
__global__ void k_apply_partition(long long, const unsigned int*, const unsigned int*, unsigned int*,
                                  const unsigned long long*, unsigned long long*, const float*, float*,
                                  const float4*, float4*);
__global__ void k_tile_flags(Tree, int, int, const BoxDesc*, const float*, const unsigned long long*,
                             unsigned int*, int);
__global__ void k_tile_table(long long, Tree, const unsigned int*, const unsigned int*, const unsigned int*,
                             const float4*, unsigned int*, Tiles, int);
__global__ void k_cell_tiles(Tree, int, const unsigned int*);
__global__ void k_box_reset(int, BoxDesc*);
__global__ void k_check_shape(int, const BoxDesc*, int, float, unsigned int*);
__global__ void k_check_build(cudaGraphConditionalHandle, const unsigned int*, const int*, int, const int*, int, int, int,
                              unsigned int, unsigned int, const unsigned long long*, int, unsigned int*);
// launchers of interact.cu
void launch_live_tasks(Engine& E, bool dens, const int* it_dev = nullptr);
void launch_density(Engine& E, const int* it_dev = nullptr, int only = -1);
void launch_gather_prep(Engine& E, const int* it_dev);
void launch_density_gather(Engine& E);
double measure_fp32_peak(cudaStream_t st, int nsm, float* scratch);
void launch_force(Engine& E);
void launch_ghost(Engine& E, int mode, int it, const int* it_dev = nullptr);
void launch_cond_keep(Engine& E, cudaGraphConditionalHandle keep);
cudaError_t add_cond_set_node(cudaGraphNode_t* node, cudaGraph_t g, const cudaGraphNode_t* deps, size_t ndeps,
                              cudaGraphConditionalHandle h, const int* flag);
void launch_iter_start(Engine& E, cudaGraphConditionalHandle iter);
void launch_iter_next(Engine& E, cudaGraphConditionalHandle iter, cudaGraphConditionalHandle force);
void launch_iter_step(Engine& E);
void launch_set_drift(Engine& E);
void launch_zero_density(Engine& E, bool all);
void launch_set_active(Engine& E);
void launch_mark_active_cells(Engine& E);
void launch_count_unconverged(Engine& E, int* out);
void launch_task_offsets(Engine& E);
void launch_task_items(Engine& E);
void launch_bracket_reset(Engine& E);
void launch_reduce(Engine& E);
void launch_save_acc(Engine& E);
void launch_kick(Engine& E);
void launch_drift(Engine& E);
void launch_set_h(Engine& E, int b, const float* src);
__global__ void k_remap_hlev(int nbox, const long long* src_tab, const int* old_lev, int* lev);
void launch_get_field(Engine& E, long long off, long long n, int field, void* out);
void launch_set_acc(Engine& E, long long off, long long n, int which, const float* src);

#define CK_PLAIN(call)                                  \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

static std::atomic<long long> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
static void count_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
long long launch_count() { return g_launches.load(std::memory_order_relaxed); }

const char* const kPhaseNames[PH_COUNT] = {"ingest",     "keys_sort",   "tree",      "lists",
                                           "shift",      "axis_sort",   "density",   "density_tasks",
                                           "ghost",      "force",       "force_tasks", "reduce",
                                           "kick_drift", "output",      "reuse"};

int Engine::prof_begin(int phase, long long* l0, cudaStream_t on) {
  *l0 = launch_count();
  if (!prof) return -1;
  if (prof_into_graph) {
    // recorded as nodes of the captured rebuild step, from events of its own
    // (created before the capture); read after every launch of the graph
    const int ev = (int)(2 * gprof_recs.size());
    if ((size_t)ev + 2 > gev_pool.size()) return -1;
    // an event node of the graph (a plain record would only order the capture)
    cudaEventRecordWithFlags(gev_pool[ev], on ? on : st, cudaEventRecordExternal);
    (void)phase;
    return ev;
  }
  while (ev_pool.size() < ev_used + 2) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return -1;
    ev_pool.push_back(e);
  }
  const int ev = (int)ev_used;
  ev_used += 2;
  cudaEventRecord(ev_pool[ev], on ? on : st);
  (void)phase;
  return ev;
}

void Engine::prof_end(int phase, int ev, long long l0, cudaStream_t on) {
  if (!prof || ev < 0) return;
  if (prof_into_graph) {
    cudaEventRecordWithFlags(gev_pool[ev + 1], on ? on : st, cudaEventRecordExternal);
    gprof_recs.push_back(GProfRec{phase, ev, launch_count() - l0});
    return;
  }
  cudaEventRecord(ev_pool[ev + 1], on ? on : st);
  prof_recs.push_back(ProfRec{phase, ev, launch_count() - l0});
}

void Engine::prof_reset() {
  prof_recs.clear();
  ev_used = 0;
  gprof_ms.assign(PH_COUNT, 0.0);
  gprof_calls.assign(PH_COUNT, 0);
  gprof_launches.assign(PH_COUNT, 0);
}

sph_status Engine::prof_read(std::vector<double>& ms, std::vector<long long>& calls, std::vector<long long>& launches) {
  ms.assign(PH_COUNT, 0.0);
  calls.assign(PH_COUNT, 0);
  launches.assign(PH_COUNT, 0);
  CK_PLAIN(cudaStreamSynchronize(st));
  for (const ProfRec& r : prof_recs) {
    float t = 0.0f;
    CK_PLAIN(cudaEventElapsedTime(&t, ev_pool[r.ev], ev_pool[r.ev + 1]));
    ms[r.phase] += t;
    calls[r.phase] += 1;
    launches[r.phase] += r.launches;
  }
  for (int k = 0; k < PH_COUNT && k < (int)gprof_ms.size(); ++k) {
    ms[k] += gprof_ms[k];
    calls[k] += gprof_calls[k];
    launches[k] += gprof_launches[k];
  }
  return SPH_OK;
}

#define CK(call)                                     \
  do {                                               \
    cudaError_t e_ = (call);                         \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

Engine::Engine(const sph_params& p, int dev, cudaStream_t s) : prm(p), device(dev), st(s) {
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device);
  if (nsm <= 0) nsm = 148;
}

Engine::~Engine() {
  drop_step_graph();
  drop_build_graph();
  for (cudaEvent_t e : gev_pool) cudaEventDestroy(e);
  for (cudaEvent_t e : ev_pool) cudaEventDestroy(e);
  if (ev_fork) cudaEventDestroy(ev_fork);
  if (ev_join) cudaEventDestroy(ev_join);
  if (st_side) cudaStreamDestroy(st_side);
}

sph_status Engine::ensure_side_stream() {
  if (st_side) return SPH_OK;
  CK(cudaEventCreateWithFlags(&ev_fork, cudaEventDisableTiming));
  CK(cudaEventCreateWithFlags(&ev_join, cudaEventDisableTiming));
  CK(cudaStreamCreateWithFlags(&st_side, cudaStreamNonBlocking));
  return SPH_OK;
}

// Every synchronisation of the engine with its stream, counted.
cudaError_t Engine::sync_stream() {
  ++host_syncs;
  return cudaStreamSynchronize(st);
}

int Engine::grid(long long work, int threads) const {
  long long g = (work + threads - 1) / threads;
  const long long cap = (long long)nsm * 16;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

sph_status Engine::cuda_fail(cudaError_t e, const char* where) {
  err = std::string("CUDA error ") + cudaGetErrorString(e) + " at " + where;
  return SPH_E_CUDA;
}

sph_status Engine::fail(sph_status s, const std::string& msg) {
  err = msg;
  return s;
}

size_t Engine::footprint_bytes() const {
  // device bytes per particle of the resident state plus the lists (estimate)
  return (size_t)N * 520 + 4096;
}

sph_status Engine::set_boxes(const std::vector<BoxSpec>& boxes) {
  spec = boxes;
  steps_in_layout = 0;
  depth_hint = 0;           // new boxes: the first build takes the full depth
  nbox = (int)boxes.size();
  off.assign(nbox + 1, 0);
  for (int b = 0; b < nbox; ++b) off[b + 1] = off[b] + boxes[b].n;
  N = off[nbox];
  hbox.assign(nbox, BoxDesc{});
  for (int b = 0; b < nbox; ++b) {
    BoxDesc& d = hbox[b];
    d.L = boxes[b].L;
    d.invL = 1.0 / boxes[b].L;
    d.margin = boxes[b].L * std::ldexp(1.0, -50);
    d.off = off[b];
    d.n = boxes[b].n;
    d.nown = boxes[b].n;
    d.periodic = boxes[b].periodic;
    int ex = 0;
    d.pow2 = std::frexp(boxes[b].L, &ex) == 0.5 ? 1u : 0u;
  }
  built = have_density = have_ghost = have_force = have_acc = false;
  reusable = false;
  n_builds = n_reuses = 0;
  sph_status s = ensure_particle_capacity();
  if (s != SPH_OK) return s;
  CK(hlev.reserve(std::max(nbox, 1)));
  CK(cudaMemsetAsync(hlev.p, 0, std::max(nbox, 1) * sizeof(int), st));
  CK(boff.reserve(nbox + 1));
  CK(cudaMemcpyAsync(boff.p, off.data(), (nbox + 1) * sizeof(long long), cudaMemcpyHostToDevice, st));
  launch_pdl(k_box_ids, grid(N), 256, st, N, nbox, boff.p, bid.p); count_launch();
  CK(sync_stream());
  return SPH_OK;
}

sph_status Engine::relayout(const std::vector<BoxSpec>& boxes, const std::vector<int>& src) {
  if (src.size() != boxes.size()) return fail(SPH_E_INVALID, "relayout: one source per box");
  long long nN = 0, maxn = 0;
  std::vector<long long> tab;   // (destination offset, source offset, count) per moved box
  for (size_t b = 0; b < boxes.size(); ++b) {
    const int sb = src[b];
    if (sb >= 0) {
      if (sb >= nbox || spec[sb].n != boxes[b].n) return fail(SPH_E_INVALID, "relayout: source box mismatch");
      tab.push_back(nN);
      tab.push_back(off[sb]);
      tab.push_back(boxes[b].n);
      maxn = std::max(maxn, boxes[b].n);
    }
    nN += boxes[b].n;
  }
  const size_t n = (size_t)std::max<long long>(nN, 1);
  CK(rl_x.reserve(3 * n));
  CK(rl_v.reserve(3 * n));
  CK(rl_m.reserve(n));
  CK(rl_u.reserve(n));
  CK(rl_h.reserve(n));
  CK(rl_hh.reserve(n));
  CK(rl_a.reserve(n));
  const int nmove = (int)(tab.size() / 3);
  if (nmove > 0) {
    CK(rl_tab.reserve(tab.size()));
    CK(cudaMemcpyAsync(rl_tab.p, tab.data(), tab.size() * sizeof(long long), cudaMemcpyHostToDevice, st));
    const dim3 g((unsigned)std::min<long long>((maxn + 255) / 256, 64), (unsigned)nmove);
    launch_pdl(k_relayout, g, 256, st, rl_tab.p, x.p, v.p, m.p, u.p, h.p, hhist.p, a_in.p, rl_x.p, rl_v.p, rl_m.p,
                                  rl_u.p, rl_h.p, rl_hh.p, rl_a.p); count_launch();
  }
  const std::vector<BoxDesc> old = hbox;
  CK(hlev_old.reserve(std::max(nbox, 1)));
  if (nbox > 0) CK(cudaMemcpyAsync(hlev_old.p, hlev.p, nbox * sizeof(int), cudaMemcpyDeviceToDevice, st));
  sph_status s = set_boxes(boxes);
  if (s != SPH_OK) return s;
  std::vector<long long> srcl(boxes.size());
  for (size_t b = 0; b < boxes.size(); ++b) {
    srcl[b] = src[b];
    if (src[b] < 0) continue;      // moved boxes keep their h history
    for (int k = 0; k < 3; ++k) hbox[b].dt_prev[k] = old[src[b]].dt_prev[k];
  }
  if (!boxes.empty()) {
    CK(hlev_src.reserve(boxes.size()));
    CK(cudaMemcpyAsync(hlev_src.p, srcl.data(), srcl.size() * sizeof(long long), cudaMemcpyHostToDevice, st));
    launch_pdl(k_remap_hlev, 1, 256, st, (int)boxes.size(), hlev_src.p, hlev_old.p, hlev.p); count_launch();
    CK(sync_stream());  // srcl is a host temporary
  }
  x.swap(rl_x);
  v.swap(rl_v);
  m.swap(rl_m);
  u.swap(rl_u);
  h.swap(rl_h);
  hhist.swap(rl_hh);
  a_in.swap(rl_a);
  return SPH_OK;
}

sph_status Engine::ensure_particle_capacity() {
  const size_t n = (size_t)std::max<long long>(N, 1);
  CK(box.reserve(std::max(nbox, 1)));
  CK(bid.reserve(n));
  CK(x.reserve(3 * n));
  CK(v.reserve(3 * n));
  CK(m.reserve(n));
  CK(u.reserve(n));
  CK(h.reserve(n));
  CK(hhist.reserve(n));
  CK(x_build.reserve(3 * n));
  CK(H_in.reserve(n));
  CK(hlo.reserve(n));
  CK(hhi.reserve(n));
  CK(conv.reserve(n));
  CK(a_in.reserve(n));
  CK(key.reserve(n));
  CK(key_tmp.reserve(n));
  CK(perm.reserve(n));
  CK(perm_tmp.reserve(n));
  CK(rs_scratch.reserve((size_t)radix_scratch_words(n)));
  CK(Hs.reserve(n));
  CK(hlimp.reserve(n));
  CK(pos4.reserve(n));
  CK(cen4.reserve(n));
  CK(vel4.reserve(n));
  CK(leaf_of.reserve(n));
  CK(top_at.reserve(n));
  CK(act.reserve(n));
  CK(Hs_tmp.reserve(n));
  CK(vel4_tmp.reserve(n));
  CK(lsrc.reserve(n));
  CK(tflag.reserve(n));
  CK(texcl.reserve(n));
  CK(tile_of.reserve(n));
  CK(tl_start.reserve(n));
  CK(tl_n.reserve(n));
  CK(tl_leaf.reserve(n));
  CK(tl_lo.reserve(n));
  CK(tl_hi.reserve(n));
  CK(tl_cen.reserve(n));
  CK(tl_active.reserve(n));
  CK(tl_changed.reserve(n));
  TL.start = tl_start.p;
  TL.n = tl_n.p;
  TL.leaf = tl_leaf.p;
  TL.lo = tl_lo.p;
  TL.hi = tl_hi.p;
  TL.cen = tl_cen.p;
  TL.active = tl_active.p;
  TL.changed = tl_changed.p;
  CK(dacc.reserve(n));
  CK(dcnt.reserve(n));
  CK(ghost4.reserve(n));
  CK(facc.reserve(n));
  CK(fvsig.reserve(n));
  CK(fcnt.reserve(n));
  CK(red.reserve(8 * std::max(nbox, 1)));
  CK(err_all.reserve(4));
  CK(pc.reserve(16));
  CK(task_ctr.reserve(4));
  CK(pk_cnt.reserve(n + 1));
  CK(pk_v.reserve(n + 1));
  CK(pk_idx.reserve(n));
  CK(pk_info.reserve(n));
  CK(pk_n.reserve(n));
  CK(pk_sums.reserve((n + 1) / 2048 + 64));
  CK(pk_tot.reserve(2));
  CK(g_n.reserve(2));
  CK(gflag.reserve(2));
  CK(dev_counters.reserve(8));
  CK(staging.reserve(24 * n));
  CK(cudaMemsetAsync(conv.p, 0, n * sizeof(int), st));
  if (cap_nodes == 0) {
    sph_status s = ensure_tree_capacity((int)std::min<long long>(std::max<long long>(4096, N / 4), 1ll << 30));
    if (s != SPH_OK) return s;
  }
  return SPH_OK;
}

sph_status Engine::ensure_tree_capacity(int nodes) {
  if (nodes <= cap_nodes && t_start.p) return SPH_OK;
  cap_nodes = nodes;
  const size_t n = (size_t)nodes;
  CK(t_start.reserve(n));
  CK(t_count.reserve(n));
  CK(t_nsmall.reserve(n));
  CK(t_axes.reserve(n));
  CK(t_sortbase.reserve(n));
  CK(t_key.reserve(n));
  CK(t_level.reserve(n));
  CK(t_box.reserve(n));
  CK(t_child.reserve(n));
  CK(t_nchild.reserve(n));
  CK(t_parent.reserve(n));
  CK(t_split.reserve(n));
  CK(t_hmax.reserve(n));
  CK(t_hlim.reserve(n));
  CK(t_cen.reserve(n));
  CK(t_active.reserve(n));
  CK(t_changed.reserve(n));
  CK(t_alo.reserve(3 * n));
  CK(t_ahi.reserve(3 * n));
  CK(t_clo.reserve(3 * n));
  CK(t_chi.reserve(3 * n));
  CK(t_tile0.reserve(n));
  CK(t_ntile.reserve(n));
  CK(t_n.reserve(8));
  T.start = t_start.p;
  T.count = t_count.p;
  T.key = t_key.p;
  T.level = t_level.p;
  T.box = t_box.p;
  T.child = t_child.p;
  T.nchild = t_nchild.p;
  T.parent = t_parent.p;
  T.split = t_split.p;
  T.hmax = t_hmax.p;
  T.nsmall = t_nsmall.p;
  T.hlim = t_hlim.p;
  T.cen = t_cen.p;
  T.axes = t_axes.p;
  T.sortbase = t_sortbase.p;
  T.active = t_active.p;
  T.changed = t_changed.p;
  T.alo = t_alo.p;
  T.ahi = t_ahi.p;
  T.clo = t_clo.p;
  T.chi = t_chi.p;
  T.tile0 = t_tile0.p;
  T.ntile = t_ntile.p;
  T.n_nodes = t_n.p;
  CK(big_node.reserve(1));
  return ensure_list_capacity(nodes, 8 * nodes, 8 * nodes);
}

sph_status Engine::ensure_list_capacity(int selfs, int pairs, int queue) {
  if (selfs > cap_self || !l_self.p) {
    cap_self = selfs;
    CK(l_self.reserve(selfs));
    CK(l_stoff.reserve(selfs + 1));
  }
  if (pairs > cap_pair || !l_pa.p) {
    cap_pair = pairs;
    CK(l_pa.reserve(pairs));
    CK(l_pb.reserve(pairs));
    CK(l_pax.reserve(pairs));
    CK(l_ptoff.reserve(pairs + 1));
  }
  CK(scan_tmp.reserve((size_t)std::max(cap_pair, cap_self) / 2048 + 64));
  if (queue > cap_queue || !q_kind[0].p) {
    cap_queue = queue;
    for (int k = 0; k < 2; ++k) {
      CK(q_kind[k].reserve(queue));
      CK(q_a[k].reserve(queue));
      CK(q_b[k].reserve(queue));
      CK(q_ax[k].reserve(queue));
    }
  }
  CK(l_counts.reserve(8));
  Lq.self_a = l_self.p;
  Lq.pair_a = l_pa.p;
  Lq.pair_b = l_pb.p;
  Lq.pair_axis = l_pax.p;
  for (int k = 0; k < 2; ++k) {
    Lq.q_kind[k] = q_kind[k].p;
    Lq.q_a[k] = q_a[k].p;
    Lq.q_b[k] = q_b[k].p;
    Lq.q_axis[k] = q_ax[k].p;
  }
  Lq.p_toff = l_ptoff.p;
  Lq.s_toff = l_stoff.p;
  Lq.counts = l_counts.p;
  return SPH_OK;
}

sph_status Engine::set_particles(int b, const double* xx, const float* vv, const float* mm, const float* uu,
                                 const float* hh, int mem) {
  if (b < 0 || b >= nbox) return fail(SPH_E_INVALID, "box index out of range");
  if (!xx || !vv || !mm || !uu || !hh) return fail(SPH_E_INVALID, "null input pointer");
  const cudaMemcpyKind kind = mem == SPH_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  const long long o = off[b], n = spec[b].n;
  CK(cudaMemcpyAsync(x.p + 3 * o, xx, 3 * n * sizeof(double), kind, st));
  CK(cudaMemcpyAsync(v.p + 3 * o, vv, 3 * n * sizeof(float), kind, st));
  CK(cudaMemcpyAsync(m.p + o, mm, n * sizeof(float), kind, st));
  CK(cudaMemcpyAsync(u.p + o, uu, n * sizeof(float), kind, st));
  const float* hsrc = hh;
  if (mem != SPH_MEM_DEVICE) {
    CK(cudaMemcpyAsync(staging.p, hh, n * sizeof(float), cudaMemcpyHostToDevice, st));
    hsrc = reinterpret_cast<const float*>(staging.p);
  }
  launch_set_h(*this, b, hsrc);      // the box keeps its h history only if h is unchanged
  CK(cudaGetLastError());
  built = have_density = have_ghost = have_force = have_acc = false;
  reusable = false;
  n_builds = n_reuses = 0;
  return SPH_OK;
}

// ----------------------------------------------------------------------- build
sph_status Engine::build() {
  for (int attempt = 0; attempt < 8; ++attempt) {
    bool retry = false;
    sph_status s = build_once(&retry);
    if (!retry) return s;
  }
  return fail(SPH_E_OOM, "decomposition lists kept overflowing");
}

static int ceil_log2(long long v) {
  int b = 0;
  while ((1ll << b) < v) ++b;
  return b;
}

sph_status Engine::build_once(bool* retry) {
  *retry = false;
  built = have_density = have_ghost = have_force = false;
  if (N == 0) return fail(SPH_E_INVALID, "no particles");
  // ---- ingest: validation, H = gamma_K h, per-box H extremes
  for (auto& d : hbox) {
    d.Hmax = 0.0f;
    d.Hmin = INFINITY;
    d.err = 0;
    d.global32 = prm.precision != 0 ? 1u : 0u;
    d.k = 0;
    d.drift2 = 0.0f;
    d.drift_u = 0.0f;
  }
  reusable = false;
  CK(cudaMemcpyAsync(box.p, hbox.data(), nbox * sizeof(BoxDesc), cudaMemcpyHostToDevice, st));
  {
    Scope sc(this, PH_INGEST);
    launch_pdl(k_ingest, grid(N), 256, st, N, bid.p, box.p, x.p, v.p, m.p, u.p, h.p, prm.gamma_kernel, H_in.p); count_launch();
  }
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(hbox.data(), box.p, nbox * sizeof(BoxDesc), cudaMemcpyDeviceToHost, st));
  CK(sync_stream());
  const int box_bits = ceil_log2(nbox);
  int dc = std::min(std::min(prm.max_depth, SPH_MAX_DEPTH), (64 - box_bits) / 3);
  int need = 0;
  kmin = 1 << 20;
  kmax = 0;
  for (int b = 0; b < nbox; ++b) {
    BoxDesc& d = hbox[b];
    if (d.err & ERR_BAD_INPUT)
      return fail(SPH_E_INVALID, "box " + std::to_string(b) + ": invalid input (NaN, h <= 0, m <= 0, u < 0 or x outside [0, L))");
    const int k0 = d.periodic ? 2 : 0;
    if (!((double)d.Hmax < std::ldexp(d.L, -k0) - d.margin))
      return fail(SPH_E_H_TOO_LARGE, "box " + std::to_string(b) + ": support radius too large for the box (periodic boxes need H < L/4)");
    // finest level whose edge clears H_max with the headroom (at least the coarsest allowed)
    const double hr = 1.0 + (double)prm.split_headroom;
    int k = k0;
    while (k + 1 <= dc && (double)d.Hmax * hr < std::ldexp(d.L, -(k + 1)) - d.margin) ++k;
    d.k = k;
    kmin = std::min(kmin, k);
    kmax = std::max(kmax, k);
    // deepest level a split can reach: more than split_frac of the cell must have H < edge/2
    const int dn = (int)std::ceil(std::log2(d.L / (double)d.Hmin)) + 1;
    need = std::max(need, dn);
  }
  // The deepest level a split could reach bounds the key width; while the boxes
  // stay the same, the previous build's deepest level plus one bounds it tighter
  // (fewer key bits to sort, fewer tree and list rounds).  A split that this bound
  // blocks sets ERR_DEPTH in the tree rounds and the build is redone at the full depth.
  const int dcap_full = std::max(std::min(dc, need), kmax);
  const bool hint = depth_hint > 0 && depth_hint_leaf == prm.leaf_max;   // a leaf size change voids it
  dcap = hint ? std::max(kmax, std::min(dcap_full, depth_hint + 1)) : dcap_full;
  const int capped = dcap < dcap_full ? 1 : 0;
  box_shift = 3 * dcap;
  key_bits = box_bits + 3 * dcap;
  CK(cudaMemcpyAsync(box.p, hbox.data(), nbox * sizeof(BoxDesc), cudaMemcpyHostToDevice, st));

  // ---- keys and sort
  long long l0;
  int ev = prof_begin(PH_SORT, &l0);
  launch_pdl(k_keys, grid(N), 256, st, N, dcap, bid.p, box.p, x.p, key.p, perm.p); count_launch();
  radix_sort(key.p, perm.p, key_tmp.p, perm_tmp.p, N, key_bits, rs_scratch.p, st);
  launch_pdl(k_gather_sorted, grid(N), 256, st, N, perm.p, H_in.p, v.p, u.p, bid.p, box.p, a_in.p, vpred, Hs.p,
                                           vel4.p); count_launch();
  prof_end(PH_SORT, ev, l0);
  CK(cudaGetLastError());

  // ---- cell tree
  ev = prof_begin(PH_TREE, &l0);
  CK(cudaMemsetAsync(t_n.p, 0, 8 * sizeof(int), st));
  CK(cudaMemsetAsync(top_at.p, 0xff, N * sizeof(int), st));
  CK(cudaMemsetAsync(err_all.p, 0, 4 * sizeof(unsigned int), st));
  launch_pdl(k_top_nodes, grid(N), 256, st, N, dcap, box_shift, box.p, key.p, T, cap_nodes, top_at.p, err_all.p); count_launch();
  launch_pdl(k_frontier_init, 1, 1, st, T, cap_nodes); count_launch();
  const int rounds = dcap - kmin + 1;
  for (int r = 0; r < rounds; ++r) {
    // with a next round, the round's last block also opens that round's frontier
    launch_pdl(k_tree_round, nsm * 8, 256, st, T, box.p, Hs.p, key.p, dcap, prm.leaf_max, prm.split_frac,
               r + 1 < rounds ? 1 : 0, capped, cap_nodes, err_all.p); count_launch();
  }
  prof_end(PH_TREE, ev, l0);
  CK(cudaGetLastError());
  // The tree's size is read before anything uses the tree: when it overflowed,
  // nodes past the last complete allocation were never written, and the build is
  // retried with more room before any kernel reads them.
  int tn[8];
  unsigned int ea[4];
  CK(cudaMemcpyAsync(tn, t_n.p, sizeof(tn), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(ea, err_all.p, sizeof(ea), cudaMemcpyDeviceToHost, st));
  CK(sync_stream());
  if (ea[0] & ERR_DEPTH) depth_hint = 0;     // the bound blocked a split: full depth
  if ((ea[0] & ERR_OVERFLOW) || tn[0] > cap_nodes) {
    sph_status s = ensure_tree_capacity(std::max(2 * cap_nodes, tn[0] + 1024));
    if (s != SPH_OK) return s;
    *retry = true;
    return SPH_OK;
  }
  if (ea[0] & ERR_DEPTH) {
    *retry = true;
    return SPH_OK;
  }
  n_nodes = tn[0];
  n_top = tn[3];
  depth_used = tn[5];
  depth_hint = tn[5];
  depth_hint_leaf = prm.leaf_max;

  // The interaction lists (on st) and the particles' leaf order, cell-relative
  // offsets and clusters (on the side stream) read the tree and nothing the other
  // writes: they run concurrently and join before the particles' H limits (which
  // read the limits the list rounds leave in the cells) and the axis sorts.  The
  // lists are enqueued first: k_items_top reads the particle keys by the pointer
  // it is given, and the leaf partition then writes a new key array in their place.
  {
    sph_status s = ensure_side_stream();
    if (s != SPH_OK) return s;
  }
  CK(cudaEventRecord(ev_fork, st));
  CK(cudaStreamWaitEvent(st_side, ev_fork, 0));
  ev = prof_begin(PH_LISTS, &l0);
  CK(cudaMemsetAsync(l_counts.p, 0, 8 * sizeof(int), st));
  launch_pdl(k_items_top, grid(13ll * n_top), 256, st, n_top, T, box.p, key.p, top_at.p, dcap, box_shift, Lq, cap_queue,
                                                  err_all.p); count_launch();
  for (int r = 0; r < rounds; ++r) {
    const int in = r & 1;
    CK(cudaMemsetAsync(l_counts.p + 2 + (in ^ 1), 0, sizeof(int), st));
    launch_pdl(k_items_expand, nsm * 8, 256, st, in, T, box.p, Lq, cap_queue, cap_self, cap_pair, err_all.p,
                                            prm.split_headroom); count_launch();
  }
  prof_end(PH_LISTS, ev, l0);
  cudaStream_t ss = st_side;
  ev = prof_begin(PH_SHIFT, &l0, ss);
  launch_pdl(k_leaves, nsm * 8, 256, ss, T, n_nodes, leaf_of.p); count_launch();
  // particles of each leaf: the ones with H above the leaf edge last (stable)
  launch_pdl(k_leaf_partition, nsm * 8, 256, ss, T, n_nodes, box.p, Hs.p, lsrc.p); count_launch();
  launch_pdl(k_apply_partition, grid(N), 256, ss, N, lsrc.p, perm.p, perm_tmp.p, key.p, key_tmp.p, Hs.p, Hs_tmp.p,
             vel4.p, vel4_tmp.p); count_launch();
  perm.swap(perm_tmp);
  key.swap(key_tmp);
  Hs.swap(Hs_tmp);
  vel4.swap(vel4_tmp);
  launch_pdl(k_shift, grid(N), 256, ss, N, box_shift, key.p, perm.p, leaf_of.p, T, box.p, x.p, m.p, Hs.p, pos4.p,
             cen4.p); count_launch();
  // clusters of at most 32 particles inside each leaf
  launch_pdl(k_tile_flags, nsm * 8, 256, ss, T, n_nodes, box_shift, box.p, Hs.p, key.p, tflag.p, prm.cluster_max);
  count_launch();
  exclusive_scan(tflag.p, texcl.p, N, rs_scratch.p, reinterpret_cast<unsigned int*>(dev_counters.p + 4), ss);
  launch_pdl(k_tile_table, grid(N), 256, ss, N, T, leaf_of.p, tflag.p, texcl.p, pos4.p, tile_of.p, TL, prm.cluster_max);
  count_launch();
  launch_pdl(k_cell_tiles, grid(n_nodes), 256, ss, T, n_nodes, tile_of.p); count_launch();
  prof_end(PH_SHIFT, ev, l0, ss);
  CK(cudaEventRecord(ev_join, ss));
  CK(cudaStreamWaitEvent(st, ev_join, 0));
  ev = prof_begin(PH_SHIFT, &l0);
  launch_pdl(k_particle_limits, grid(N), 256, st, N, T, leaf_of.p, hlimp.p); count_launch();
  prof_end(PH_SHIFT, ev, l0);

  // ---- sorted projections
  CK(big_count.reserve(1));
  if (cap_big == 0) {
    cap_big = 4096;
    CK(big_node.reserve(cap_big));
    CK(big_axis.reserve(cap_big));
    CK(big_off.reserve(cap_big));
  }
  ev = prof_begin(PH_AXIS_SORT, &l0);
  CK(cudaMemsetAsync(big_count.p, 0, sizeof(unsigned long long), st));
  CK(mid_seg.reserve(13 * (size_t)std::max(n_nodes, 1)));
  CK(mid_count.reserve(1));
  CK(cudaMemsetAsync(mid_count.p, 0, sizeof(unsigned int), st));
  launch_pdl(k_mark_axes, nsm * 8, 256, st, Lq, cap_pair, T); count_launch();
  launch_pdl(k_sort_alloc, grid(n_nodes), 256, st, T, n_nodes, Lq, big_node.p, big_axis.p, big_off.p, big_count.p,
             cap_big, mid_seg.p, mid_count.p, 0xffffffffu, 0xffffffffu, err_all.p); count_launch();
  launch_task_offsets(*this);
  prof_end(PH_AXIS_SORT, ev, l0);
  CK(cudaGetLastError());
  int lc[8];
  unsigned long long bcw = 0;
  CK(cudaMemcpyAsync(lc, l_counts.p, sizeof(lc), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(&bcw, big_count.p, sizeof(bcw), cudaMemcpyDeviceToHost, st));
  unsigned int ntl = 0;
  CK(cudaMemcpyAsync(&ntl, dev_counters.p + 4, sizeof(ntl), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(ea, err_all.p, sizeof(ea), cudaMemcpyDeviceToHost, st));
  CK(sync_stream());
  const int last_q = lc[2 + (rounds & 1)];
  if ((ea[0] & ERR_OVERFLOW) || lc[0] > cap_self || lc[1] > cap_pair || last_q != 0) {
    sph_status s = ensure_list_capacity(std::max(cap_self, lc[0]) * 2, std::max(cap_pair, lc[1]) * 2,
                                        cap_queue * 2);
    if (s != SPH_OK) return s;
    *retry = true;
    return SPH_OK;
  }
  const long long bc[2] = {(long long)(bcw >> 40), (long long)(bcw & ((1ull << 40) - 1ull))};
  if (bc[0] > cap_big) {
    cap_big = (int)(2 * bc[0]);
    CK(big_node.reserve(cap_big));
    CK(big_axis.reserve(cap_big));
    CK(big_off.reserve(cap_big));
    *retry = true;
    return SPH_OK;
  }
  n_tiles = ntl;
  n_selfs = lc[0];
  n_pairs = lc[1];
  n_segments = lc[4];
  n_entries = (unsigned int)lc[5];
  n_big = (int)bc[0];
  n_big_entries = bc[1];
  CK(l_ptask.reserve(std::max(lc[6], 1)));
  CK(l_stask.reserve(std::max(lc[7], 1)));
  CK(l_plive.reserve(std::max(lc[6] + lc[7], 1)));
  CK(g_live.reserve(l_plive.n));
  CK(l_nlive.reserve(1));
  n_ptasks = lc[6];
  n_stasks = lc[7];
  Lq.p_task = l_ptask.p;
  Lq.s_task = l_stask.p;
  Lq.p_live = l_plive.p;
  Lq.n_live = l_nlive.p;
  launch_task_items(*this);
  CK(sort_r.reserve(std::max<long long>(n_entries, 1)));
  CK(sort_i.reserve(std::max<long long>(n_entries, 1)));
  ev = prof_begin(PH_AXIS_SORT, &l0);
  if (prm.sort_merge)
    launch_pdl(k_sort_merge, nsm * 8, 256, st, mid_seg.p, mid_count.p, T, TL, sort_r.p, sort_i.p);
  else
    launch_pdl(k_sort_small, nsm * 8, 256, st, mid_seg.p, mid_count.p, T, TL, sort_r.p, sort_i.p);
  count_launch();
  if (n_big > 0) {
    const size_t nb = (size_t)n_big_entries;
    CK(ckey.reserve(nb));
    CK(ckey_tmp.reserve(nb));
    CK(cval.reserve(nb));
    CK(cval_tmp.reserve(nb));
    if (rs_scratch.n < (size_t)radix_scratch_words(nb)) CK(rs_scratch.reserve(radix_scratch_words(nb)));
    launch_pdl(k_sort_big_keys, std::min(n_big, nsm * 8), 256, st, n_big, big_node.p, big_axis.p, big_off.p, T, TL,
               ckey.p, cval.p, big_count.p, cap_big); count_launch();
    radix_sort(ckey.p, cval.p, ckey_tmp.p, cval_tmp.p, (long long)nb, 32 + std::max(1, ceil_log2(n_big)),
               rs_scratch.p, st);
    launch_pdl(k_sort_big_scatter, std::min(n_big, nsm * 8), 256, st, n_big, big_node.p, big_axis.p, big_off.p, T, TL,
               cval.p, sort_r.p, sort_i.p, big_count.p, cap_big); count_launch();
  }
  prof_end(PH_AXIS_SORT, ev, l0);
  CK(cudaGetLastError());
  built = true;
  // positions of this decomposition, for the displacement test of a later reuse
  CK(cudaMemcpyAsync(x_build.p, x.p, 3 * N * sizeof(double), cudaMemcpyDeviceToDevice, st));
  reusable = true;
  ++n_builds;
  rec_valid = false;        // the records name this build's tasks
  graph_ready = false;      // a captured step holds this build's sizes and buffers
  bgraph_ready = false;     // ... and so does the captured rebuild step (the buffers swapped)
  gb_last_q = 2 + (rounds & 1);
  return SPH_OK;
}

// ----------------------------------------------------------------------- passes
// The pool holds the last recordings' need with a quarter to spare, and at least
// 1.5 batches per particle (clustered boxes take about one).  A recording that
// runs out keeps the tasks it completed; the others take the full force path.
// A larger pool moves the buffers, so the captured steps are captured again.
sph_status Engine::rec_prepare() {
  if (!prm.pair_cache) return SPH_OK;
  if (rec_unread && rec_ctr.p) {
    // the last recording's need was not read back with a synchronisation of its own
    unsigned int rc = 0;
    CK(cudaMemcpyAsync(&rc, rec_ctr.p, sizeof(rc), cudaMemcpyDeviceToHost, st));
    CK(sync_stream());
    rec_used = rc;
    rec_need = std::max<long long>(rec_need, rc);
  }
  rec_unread = false;
  long long want = std::max<long long>(rec_need + rec_need / 4, (N + N / 2) / REC_CHUNK) + 64;
  want = std::min<long long>(want, (long long)(REC_NONE / REC_CHUNK) - 1);
  bool moved = false;
  if ((size_t)want > rec_next.n || !rec_pool.p) {
    rec_pool.release();
    rec_next.release();
    moved = true;
    if (rec_pool.reserve((size_t)want * REC_CHUNK * 64) != cudaSuccess ||
        rec_next.reserve((size_t)want) != cudaSuccess) {
      // no room for the records: the force pass culls on its own
      cudaGetLastError();
      rec_pool.release();
      rec_next.release();
      R = PairRec{};
      if (!gcap) graph_ready = bgraph_ready = false;
      return SPH_OK;
    }
  }
  CK(rec_ctr.reserve(1));
  const size_t np = std::max<size_t>(l_ptask.n, 1), ns = std::max<size_t>(l_stask.n, 1);
  if (np > rec_pt.n || ns > rec_st.n) moved = true;
  CK(rec_pt.reserve(np));
  CK(rec_st.reserve(ns));
  R.pool = rec_pool.p;
  R.next = rec_next.p;
  R.ctr = rec_ctr.p;
  R.ptask = rec_pt.p;
  R.stask = rec_st.p;
  R.cap = (unsigned int)(rec_next.n);
  if (moved && !gcap) {
    graph_ready = false;
    bgraph_ready = false;
  }
  return SPH_OK;
}

void Engine::rec_enqueue_reset() {
  rec_valid = false;
  if (!prm.pair_cache || !rec_pool.p) return;
  const size_t np = gcap ? rec_pt.n : (size_t)n_ptasks, ns = gcap ? rec_st.n : (size_t)n_stasks;
  const size_t nn = gcap ? (size_t)cap_nodes : (size_t)n_nodes, nt = gcap ? (size_t)N : (size_t)n_tiles;
  cudaMemsetAsync(rec_ctr.p, 0, sizeof(unsigned int), st);
  if (np) cudaMemsetAsync(rec_pt.p, 0xff, np * sizeof(uint2), st);
  if (ns) cudaMemsetAsync(rec_st.p, 0xff, ns * sizeof(uint2), st);
  if (nn) {
    cudaMemsetAsync(t_changed.p, 0, nn, st);
    cudaMemsetAsync(t_clo.p, 0xff, 3 * nn * sizeof(unsigned int), st);
    cudaMemsetAsync(t_chi.p, 0, 3 * nn * sizeof(unsigned int), st);
  }
  if (nt) cudaMemsetAsync(tl_changed.p, 0, nt, st);
  rec_valid = true;
  rec_unread = true;
}

sph_status Engine::set_all_active() {
  launch_set_active(*this);
  CK(cudaGetLastError());
  return SPH_OK;
}

sph_status Engine::density_pass() {
  {
    Scope sc(this, PH_DENSITY_TASKS);
    launch_zero_density(*this, false);
    launch_live_tasks(*this, true);
  }
  {
    Scope sc(this, PH_DENSITY);
    launch_density(*this);
  }
  CK(cudaGetLastError());
  return SPH_OK;
}

sph_status Engine::density() {
  if (!built) {
    sph_status s = build();
    if (s != SPH_OK) return s;
  }
  if (count_pairs) CK(cudaMemsetAsync(pc.p, 0, 16 * sizeof(unsigned long long), st));
  sph_status s = set_all_active();
  if (s != SPH_OK) return s;
  s = rec_prepare();
  if (s != SPH_OK) return s;
  rec_enqueue_reset();
  s = density_pass();
  if (s != SPH_OK) return s;
  CK(cudaMemsetAsync(dev_counters.p, 0, 4 * sizeof(int), st));
  {
    Scope sc(this, PH_GHOST);
    launch_ghost(*this, 0, 1);
  }
  CK(cudaGetLastError());
  have_density = have_ghost = true;
  have_force = false;
  last_iters = 1;
  last_rebuilds = 0;
  last_gathered = 0;
  return SPH_OK;
}

sph_status Engine::h_update(long long* n_unconverged, int* iterations) {
  if (!built) {
    sph_status s = build();
    if (s != SPH_OK) return s;
  }
  if (count_pairs) CK(cudaMemsetAsync(pc.p, 0, 16 * sizeof(unsigned long long), st));
  launch_bracket_reset(*this);
  sph_status s = set_all_active();
  if (s != SPH_OK) return s;
  s = rec_prepare();
  if (s != SPH_OK) return s;
  rec_enqueue_reset();
  // Iterations run in batches launched without a host round trip: the iteration
  // counter and the stopping test live on the device (k_iter_step), and the
  // kernels of iterations launched past a stop return at once.  One
  // synchronisation per batch reads where the iteration stands.
  constexpr int H_BATCH = 2;
  int it = 1, rebuilds = 0;
  CK(it_dev.reserve(4));
  CK(cudaMemsetAsync(dev_counters.p, 0, 4 * sizeof(int), st));
  CK(cudaMemsetAsync(err_all.p, 0, 4 * sizeof(unsigned int), st));
  int itv[3] = {1, 0, 0};
  CK(cudaMemcpyAsync(it_dev.p, itv, 3 * sizeof(int), cudaMemcpyHostToDevice, st));
  CK(cudaMemsetAsync(g_n.p + 1, 0, sizeof(unsigned int), st));
  unsigned int ngath = 0;
  bool fresh = true;      // all particles marked active (first iteration, or after a rebuild)
  for (;;) {
    const int nb = std::min(H_BATCH, prm.h_max_iter - it + 1);
    for (int k = 0; k < nb; ++k) {
      if (!fresh) launch_mark_active_cells(*this);
      fresh = false;
      {
        Scope sc(this, PH_DENSITY_TASKS);
        launch_zero_density(*this, false);
        if (it + k > 1) launch_gather_prep(*this, it_dev.p);
        launch_live_tasks(*this, true, it_dev.p);
      }
      {
        // iteration it + k unless the iteration stopped earlier in the batch (its
        // kernels then find no tasks): the pass kind is known here
        Scope sc(this, PH_DENSITY);
        launch_density(*this, it_dev.p, it + k > 1 ? 1 : 0);
        if (it + k > 1) launch_density_gather(*this);
      }
      {
        Scope sc(this, PH_GHOST);
        launch_ghost(*this, 1, 0, it_dev.p);
        launch_iter_step(*this);
      }
    }
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(itv, it_dev.p, 3 * sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(&ngath, g_n.p + 1, sizeof(unsigned int), cudaMemcpyDeviceToHost, st));
    unsigned int rc = 0;
    const bool read_rec = rebuilds == 0 && it == 1 && rec_valid;
    if (read_rec) CK(cudaMemcpyAsync(&rc, rec_ctr.p, sizeof(rc), cudaMemcpyDeviceToHost, st));
    CK(sync_stream());
    if (read_rec) {
      rec_used = rc;
      rec_need = std::max<long long>(rec_need, rc);
      rec_unread = false;
    }
    if (rebuilds == 0 && it == 1) first_active = itv[1];
    it = itv[0];
    if (itv[2] == 1) break;            // every particle finalised (at the limit, unconverged ones too)
    if (itv[2] == 2) {
      s = build();   // the input-order h carries the iteration's state
      if (s != SPH_OK) return s;
      s = set_all_active();
      if (s != SPH_OK) return s;
      ++rebuilds;
      if (it >= prm.h_max_iter) break;
      ++it;
      itv[0] = it;
      itv[2] = 0;
      CK(cudaMemcpyAsync(it_dev.p, itv, 3 * sizeof(int), cudaMemcpyHostToDevice, st));
      CK(cudaMemsetAsync(err_all.p, 0, 4 * sizeof(unsigned int), st));
      CK(cudaMemsetAsync(dev_counters.p, 0, 4 * sizeof(int), st));
      fresh = true;
      continue;
    }
    if (it >= prm.h_max_iter) break;   // not reached: the step stops at the limit
    // itv[2] == 0: the batch ran and more iterations are needed (it_dev[0] advanced)
  }
  if (it > prm.h_max_iter) it = prm.h_max_iter;
  // particles that never converged: the last iteration finalises them with their
  // flag cleared, so they are counted whenever the iteration ran to its limit
  long long nu = 0;
  if (it == prm.h_max_iter) {
    int cnt = 0;
    CK(cudaMemsetAsync(dev_counters.p + 1, 0, sizeof(int), st));
    launch_count_unconverged(*this, dev_counters.p + 1);
    CK(cudaMemcpyAsync(&cnt, dev_counters.p + 1, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(sync_stream());
    nu = cnt;
  }
  last_iters = it;
  last_rebuilds = rebuilds;
  last_gathered = ngath;
  last_unconverged = nu;
  if (n_unconverged) *n_unconverged = nu;
  if (iterations) *iterations = it;
  have_density = have_ghost = true;
  have_force = false;
  if (nu > 0) return fail(SPH_E_NOT_CONVERGED, std::to_string(nu) + " particles did not converge");
  return SPH_OK;
}

sph_status Engine::force() {
  if (!have_ghost) return fail(SPH_E_NOT_BUILT, "force pass needs a density pass first");
  CK(cudaMemsetAsync(facc.p, 0, N * sizeof(float4), st));
  CK(cudaMemsetAsync(fvsig.p, 0, N * sizeof(float), st));
  if (count_pairs) CK(cudaMemsetAsync(fcnt.p, 0, N * sizeof(unsigned int), st));
  {
    Scope sc(this, PH_FORCE_TASKS);
    launch_live_tasks(*this, false);
  }
  {
    Scope sc(this, PH_FORCE);
    launch_force(*this);
  }
  {
    Scope sc(this, PH_REDUCE);
    launch_reduce(*this);
    launch_save_acc(*this);
  }
  CK(cudaGetLastError());
  have_force = true;
  have_acc = true;
  have_fcount = count_pairs;
  return SPH_OK;
}

sph_status Engine::upload_boxes() {
  CK(cudaMemcpyAsync(box.p, hbox.data(), nbox * sizeof(BoxDesc), cudaMemcpyHostToDevice, st));
  return SPH_OK;
}

sph_status Engine::step(double dt) {
  for (auto& d : hbox) d.dt = dt;
  return step_boxes();
}

// Weights of the last l + 1 roots of N~(h) = N_ngb (l = 1..3, row l of hw), at
// times 0, -dt_prev[0], -dt_prev[0] - dt_prev[1], ..., in the polynomial through
// them evaluated at dt (Lagrange form).  The level l of a box lives on the device.
static void root_weights(BoxDesc& d) {
  double T[4] = {0.0, 0.0, 0.0, 0.0};
  for (int k = 1; k < 4; ++k) T[k] = T[k - 1] - d.dt_prev[k - 1];
  for (int l = 0; l < 4; ++l) {
    const int n = l + 1;
    for (int i = 0; i < 4; ++i) {
      double w = i < n ? 1.0 : 0.0;
      for (int j = 0; j < n && i < n; ++j)
        if (j != i) w *= (d.dt - T[j]) / (T[i] - T[j]);
      d.hw[l][i] = (float)w;
    }
  }
}

sph_status Engine::step_boxes() {
  for (auto& d : hbox)
    if (d.dt > 0.0) root_weights(d);
  vpred = 0;
  const sph_status s = step_boxes_once();
  vpred = 0;
  const bool done = s == SPH_OK || s == SPH_E_NOT_CONVERGED;
  for (auto& d : hbox) {
    // the drift shifted the history; this step's ghost pass wrote its root
    if (d.dt > 0.0) {
      d.dt_prev[2] = d.dt_prev[1];
      d.dt_prev[1] = d.dt_prev[0];
      d.dt_prev[0] = d.dt;
    }
  }
  if (!done && nbox > 0) cudaMemsetAsync(hlev.p, 0, nbox * sizeof(int), st);   // restart every history
  return s;
}

// Kick-drift-kick (Section III-B: fixed time step, forces on all particles every
// step): v += a dt/2, u += du/dt dt/2 with the forces of the previous step, x +=
// v dt in FP64, then build, density with h iteration, force and reductions at
// the new positions, and the closing half kick.  Boxes with dt = 0 only run the
// passes.  The first call computes the starting forces.
sph_status Engine::step_boxes_once() {
  sph_status s;
  bool moving = false;
  for (auto& d : hbox) moving |= d.dt > 0.0;
  if (moving && !have_acc) {
    s = build();
    if (s != SPH_OK) return s;
    s = h_update(nullptr, nullptr);
    if (s != SPH_OK && s != SPH_E_NOT_CONVERGED) return s;
    s = force();
    if (s != SPH_OK) return s;
  }
  if (moving && prm.reuse && reusable && !prof && !count_pairs && !graph_off && prm.graphs) {
    // the whole step, kick and drift included, as one captured graph
    s = upload_boxes();
    if (s != SPH_OK) return s;
    vpred = 1;
    return step_graph();
  }
  if (moving) ++steps_in_layout;
  if (moving && !prm.reuse && built && !count_pairs && !graph_off && prm.graphs && steps_in_layout > 2) {
    // a step that rebuilds, as one captured graph (captured again after every
    // host-driven build: the graph holds that build's shape and capacities)
    s = upload_boxes();
    if (s != SPH_OK) return s;
    vpred = 1;
    return build_step_graph();
  }
  if (moving) {
    s = upload_boxes();
    if (s != SPH_OK) return s;
    {
      Scope sc(this, PH_STEP);
      launch_kick(*this);
      launch_drift(*this);
    }
    CK(cudaGetLastError());
    vpred = 1;
  }
  return step_host(moving);
}

// The rest of a step after its kick and drift: build (or keep) the decomposition,
// the h iteration, the force pass and the closing kick, host-sequenced.
sph_status Engine::step_host(bool moving) {
  ++steps_host;
  sph_status s = reuse_or_build();
  if (s != SPH_OK) return s;
  sph_status hs = h_update(nullptr, nullptr);
  if (hs != SPH_OK && hs != SPH_E_NOT_CONVERGED) return hs;
  s = force();
  if (s != SPH_OK) return s;
  if (moving) {
    Scope sc(this, PH_STEP);
    launch_kick(*this);
    CK(cudaGetLastError());
  }
  return hs;
}

// Decomposition reuse over steps (Section II-C: the sorted indices are re-used
// until the decomposition must be re-computed).  The decomposition is kept when
// every particle's H plus twice its box's largest displacement since the build
// stays below the limit its interactions assumed: a pair within H was then at
// most H + 2 d apart when its cells were assigned, so it is still covered by
// exactly one interaction.  Particles keep their cells, clusters and sorted
// indices; offsets, velocities, cluster boxes and cell H maxima are refreshed,
// and the sweeps widen their tests by the displacement.
sph_status Engine::reuse_or_build() {
  if (!prm.reuse || !reusable) return build();
  long long l0;
  const int ev = prof_begin(PH_REUSE, &l0);
  CK(dmax_bits.reserve(nbox));
  CK(reuse_flag.reserve(1));
  CK(cudaMemsetAsync(dmax_bits.p, 0, nbox * sizeof(unsigned long long), st));
  CK(cudaMemsetAsync(reuse_flag.p, 0, sizeof(unsigned int), st));
  launch_pdl(k_displacement, grid(N), 256, st, N, bid.p, box.p, x.p, x_build.p, dmax_bits.p); count_launch();
  launch_pdl(k_reuse_limits, grid(N), 256, st, N, box_shift, key.p, T, leaf_of.p, perm.p, h.p, prm.gamma_kernel,
                                          dmax_bits.p, hlimp.p, reuse_flag.p); count_launch();
  std::vector<unsigned long long> dm(nbox);
  unsigned int flag = 0;
  CK(cudaMemcpyAsync(dm.data(), dmax_bits.p, nbox * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(&flag, reuse_flag.p, sizeof(unsigned int), cudaMemcpyDeviceToHost, st));
  CK(sync_stream());
  if (flag) {
    prof_end(PH_REUSE, ev, l0);
    return build();
  }
  for (int b = 0; b < nbox; ++b) {
    double d;
    std::memcpy(&d, &dm[b], sizeof(d));
    hbox[b].drift2 = (float)(2.0 * d);
    hbox[b].drift_u = (float)(d / hbox[b].L);
  }
  CK(cudaMemcpyAsync(box.p, hbox.data(), nbox * sizeof(BoxDesc), cudaMemcpyHostToDevice, st));
  launch_pdl(k_ingest, grid(N), 256, st, N, bid.p, box.p, x.p, v.p, m.p, u.p, h.p, prm.gamma_kernel, H_in.p); count_launch();
  launch_pdl(k_gather_sorted, grid(N), 256, st, N, perm.p, H_in.p, v.p, u.p, bid.p, box.p, a_in.p, vpred, Hs.p,
                                           vel4.p); count_launch();
  launch_pdl(k_shift, grid(N), 256, st, N, box_shift, key.p, perm.p, leaf_of.p, T, box.p, x.p, m.p, Hs.p, pos4.p, cen4.p); count_launch();
  CK(cudaMemsetAsync(t_hmax.p, 0, n_nodes * sizeof(float), st));
  launch_pdl(k_leaf_hmax, nsm * 8, 256, st, T, n_nodes, Hs.p); count_launch();
  launch_pdl(k_tile_boxes, grid(32 * n_tiles), 256, st, n_tiles, TL, pos4.p); count_launch();
  prof_end(PH_REUSE, ev, l0);
  CK(cudaGetLastError());
  built = true;
  have_density = have_ghost = have_force = false;
  ++n_reuses;
  return SPH_OK;
}

// ------------------------------------------------------------ captured step
// A step that keeps the decomposition, as one CUDA graph with conditional nodes:
//   kick, drift, the displacement test (a child graph), then
//   IF the decomposition stays: refresh offsets, velocities, boxes and H maxima,
//     and set the h iteration up;
//   WHILE particles still iterate (no rebuild needed, limit not reached): one
//     density pass and its h update, the iteration counter kept on the device;
//   IF the iteration ended without a rebuild: force pass, reductions, the saved
//     accelerations and the closing kick.
// One synchronisation at the end reads what happened: when the test failed or an
// iteration needed a rebuild, the host completes the step with a full build.
void Engine::drop_step_graph() {
  if (step_x) cudaGraphExecDestroy(step_x);
  if (step_g) cudaGraphDestroy(step_g);
  step_x = nullptr;
  step_g = nullptr;
  graph_ready = false;
}

#define CKG(call)                                                                  \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess) {                                                       \
      cudaStreamCaptureStatus cs_;                                                 \
      if (cudaStreamIsCapturing(st, &cs_) == cudaSuccess && cs_ != cudaStreamCaptureStatusNone) { \
        cudaGraph_t g_;                                                            \
        cudaStreamEndCapture(st, &g_);                                             \
        if (g_) cudaGraphDestroy(g_);                                              \
      }                                                                            \
      cudaGetLastError();                                                          \
      drop_step_graph();                                                           \
      graph_off = true;                                                            \
      return fail(SPH_E_CUDA, std::string("step capture: ") + cudaGetErrorString(e_)); \
    }                                                                              \
  } while (0)

sph_status Engine::capture_step_graph() {
  drop_step_graph();
  {
    const sph_status rs = rec_prepare();
    if (rs != SPH_OK) return rs;
  }
  CK(dmax_bits.reserve(nbox));
  CK(reuse_flag.reserve(1));
  CK(it_dev.reserve(4));
  const long long c0 = launch_count();
  const cudaStreamCaptureMode mode = cudaStreamCaptureModeThreadLocal;
  CKG(cudaGraphCreate(&step_g, 0));
  cudaGraphConditionalHandle keep, iter, frc;
  CKG(cudaGraphConditionalHandleCreate(&keep, step_g, 0, cudaGraphCondAssignDefault));
  CKG(cudaGraphConditionalHandleCreate(&iter, step_g, 0, cudaGraphCondAssignDefault));
  CKG(cudaGraphConditionalHandleCreate(&frc, step_g, 0, cudaGraphCondAssignDefault));
  // kick, drift, displacement test
  cudaGraph_t g1 = nullptr;
  CKG(cudaStreamBeginCapture(st, mode));
  launch_kick(*this);
  launch_drift(*this);
  CKG(cudaMemsetAsync(dmax_bits.p, 0, nbox * sizeof(unsigned long long), st));
  CKG(cudaMemsetAsync(reuse_flag.p, 0, sizeof(unsigned int), st));
  launch_pdl(k_displacement, grid(N), 256, st, N, bid.p, box.p, x.p, x_build.p, dmax_bits.p); count_launch();
  launch_pdl(k_reuse_limits, grid(N), 256, st, N, box_shift, key.p, T, leaf_of.p, perm.p, h.p, prm.gamma_kernel,
                                          dmax_bits.p, hlimp.p, reuse_flag.p); count_launch();
  launch_set_drift(*this);
  launch_cond_keep(*this, keep);
  CKG(cudaStreamEndCapture(st, &g1));
  g_pre = launch_count() - c0;
  cudaGraphNode_t n1, n2, n3, n4;
  CKG(cudaGraphAddChildGraphNode(&n1, step_g, nullptr, 0, g1));
  cudaGraphDestroy(g1);
  // IF kept: refresh and set the iteration up
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = keep;
  cp.conditional.type = cudaGraphCondTypeIf;
  cp.conditional.size = 1;
  CKG(cudaGraphAddNode(&n2, step_g, &n1, nullptr, 1, &cp));
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  long long c1 = launch_count();
  CKG(cudaStreamBeginCaptureToGraph(st, body, nullptr, nullptr, 0, mode));
  launch_pdl(k_ingest, grid(N), 256, st, N, bid.p, box.p, x.p, v.p, m.p, u.p, h.p, prm.gamma_kernel, H_in.p); count_launch();
  launch_pdl(k_gather_sorted, grid(N), 256, st, N, perm.p, H_in.p, v.p, u.p, bid.p, box.p, a_in.p, vpred, Hs.p,
                                           vel4.p); count_launch();
  launch_pdl(k_shift, grid(N), 256, st, N, box_shift, key.p, perm.p, leaf_of.p, T, box.p, x.p, m.p, Hs.p, pos4.p, cen4.p); count_launch();
  CKG(cudaMemsetAsync(t_hmax.p, 0, n_nodes * sizeof(float), st));
  launch_pdl(k_leaf_hmax, nsm * 8, 256, st, T, n_nodes, Hs.p); count_launch();
  launch_pdl(k_tile_boxes, grid(32 * n_tiles), 256, st, n_tiles, TL, pos4.p); count_launch();
  launch_bracket_reset(*this);
  launch_set_active(*this);
  CKG(cudaMemsetAsync(dev_counters.p, 0, 4 * sizeof(int), st));
  CKG(cudaMemsetAsync(err_all.p, 0, 4 * sizeof(unsigned int), st));
  rec_enqueue_reset();
  launch_iter_start(*this, iter);
  CKG(cudaStreamEndCapture(st, &body));
  g_keep = launch_count() - c1;
  // WHILE iterating: one density pass and its h update
  cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = iter;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  CKG(cudaGraphAddNode(&n3, step_g, &n2, nullptr, 1, &cp));
  body = cp.conditional.phGraph_out[0];
  c1 = launch_count();
  CKG(cudaStreamBeginCaptureToGraph(st, body, nullptr, nullptr, 0, mode));
  launch_zero_density(*this, false);
  launch_gather_prep(*this, it_dev.p);
  launch_live_tasks(*this, true, it_dev.p);
  launch_density(*this, it_dev.p);
  launch_density_gather(*this);
  launch_ghost(*this, 1, 0, it_dev.p);
  launch_iter_next(*this, iter, frc);
  launch_mark_active_cells(*this);
  CKG(cudaStreamEndCapture(st, &body));
  g_iter = launch_count() - c1;
  // IF finished without a rebuild: force pass and the closing kick
  cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = frc;
  cp.conditional.type = cudaGraphCondTypeIf;
  cp.conditional.size = 1;
  CKG(cudaGraphAddNode(&n4, step_g, &n3, nullptr, 1, &cp));
  body = cp.conditional.phGraph_out[0];
  c1 = launch_count();
  CKG(cudaStreamBeginCaptureToGraph(st, body, nullptr, nullptr, 0, mode));
  CKG(cudaMemsetAsync(facc.p, 0, N * sizeof(float4), st));
  CKG(cudaMemsetAsync(fvsig.p, 0, N * sizeof(float), st));
  launch_live_tasks(*this, false);
  launch_force(*this);
  launch_reduce(*this);
  launch_save_acc(*this);
  launch_kick(*this);
  CKG(cudaStreamEndCapture(st, &body));
  g_force = launch_count() - c1;
  CKG(cudaGraphInstantiate(&step_x, step_g, 0));
  count_launches(-(launch_count() - c0));     // capturing launches nothing
  graph_ready = true;
  return SPH_OK;
}

sph_status Engine::step_graph() {
  if (!graph_ready) {
    sph_status s = capture_step_graph();
    if (s != SPH_OK) return s;
  }
  CK(cudaGraphLaunch(step_x, st));
  unsigned int flag = 0, ea = 0, rc = 0;
  int itv[2] = {0, 0};
  CK(cudaMemcpyAsync(&flag, reuse_flag.p, sizeof(flag), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(&ea, err_all.p, sizeof(ea), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(itv, it_dev.p, sizeof(itv), cudaMemcpyDeviceToHost, st));
  if (R.pool) CK(cudaMemcpyAsync(&rc, rec_ctr.p, sizeof(rc), cudaMemcpyDeviceToHost, st));
  CK(sync_stream());
  if (R.pool && !flag) {
    rec_used = rc;
    rec_need = std::max<long long>(rec_need, rc);
    rec_unread = false;
  }
  const bool rebuild = flag != 0 || (ea & ERR_REBUILD) != 0u;
  count_launches(g_pre + (flag ? 0 : g_keep + (long long)itv[0] * g_iter + (rebuild ? 0 : g_force)));
  if (rebuild) {
    // kick and drift are done: complete the step with a full build
    sph_status s = build();
    if (s != SPH_OK) return s;
    sph_status hs = h_update(nullptr, nullptr);
    if (hs != SPH_OK && hs != SPH_E_NOT_CONVERGED) return hs;
    s = force();
    if (s != SPH_OK) return s;
    launch_kick(*this);
    CK(cudaGetLastError());
    return hs;
  }
  ++n_reuses;
  built = true;
  have_density = have_ghost = have_force = have_acc = true;
  rec_valid = R.pool != nullptr;
  last_iters = itv[0];
  last_rebuilds = 0;
  last_gathered = 0;
  first_active = itv[1];
  long long nu = 0;
  if (itv[0] >= prm.h_max_iter) {
    int cnt = 0;
    CK(cudaMemsetAsync(dev_counters.p + 1, 0, sizeof(int), st));
    launch_count_unconverged(*this, dev_counters.p + 1);
    CK(cudaMemcpyAsync(&cnt, dev_counters.p + 1, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(sync_stream());
    nu = cnt;
  }
  last_unconverged = nu;
  if (nu > 0) return fail(SPH_E_NOT_CONVERGED, std::to_string(nu) + " particles did not converge");
  return SPH_OK;
}

// ------------------------------------------------------------ captured rebuild step
// A step that rebuilds the decomposition (the default protocol), as one CUDA
// graph with conditional nodes:
//   the kick and the drift, then the whole build, every launch sized by the
//   capacities of the last host-driven build and reading this build's counts on
//   the device; k_check_shape flags a box whose support radii no longer give the
//   top level that build chose, the tree rounds flag a split that the depth
//   bound blocks, and k_check_build checks every count against its capacity;
//   IF the build held: the h iteration set up;
//   WHILE particles still iterate (no rebuild needed, limit not reached): one
//   density pass and its h update, the iteration counter kept on the device;
//   IF the iteration ended without a rebuild: force pass, reductions, the saved
//   accelerations and the closing kick.
// One synchronisation at the end reads what happened.  When the build did not
// hold or an iteration needed a rebuild, the host completes the step (kick and
// drift are done) with a host-driven build; that build drops the graph, and the
// next step captures it again with the new build's shape and capacities.  The
// capture reserves every buffer first (nothing can be allocated while capturing)
// and swaps the double buffers of the particle side exactly as a build does, so
// that every launch of the graph leaves the data where the host expects it.
void Engine::drop_build_graph() {
  if (bstep_x) cudaGraphExecDestroy(bstep_x);
  if (bstep_g) cudaGraphDestroy(bstep_g);
  bstep_x = nullptr;
  bstep_g = nullptr;
  bgraph_ready = false;
  gprof_recs.clear();
}

#define CKB(call)                                                                  \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess) {                                                       \
      cudaStreamCaptureStatus cs_;                                                 \
      if (cudaStreamIsCapturing(st, &cs_) == cudaSuccess && cs_ != cudaStreamCaptureStatusNone) { \
        cudaGraph_t g_;                                                            \
        cudaStreamEndCapture(st, &g_);                                             \
        if (g_) cudaGraphDestroy(g_);                                              \
      }                                                                            \
      cudaGetLastError();                                                          \
      gcap = false;                                                                \
      prof_into_graph = false;                                                     \
      drop_build_graph();                                                          \
      graph_off = true;                                                            \
      return fail(SPH_E_CUDA, std::string("rebuild step capture: ") + cudaGetErrorString(e_)); \
    }                                                                              \
  } while (0)

// The build of a captured rebuild step (enqueued while capturing; gcap set).
sph_status Engine::enqueue_captured_build() {
  CKB(cudaMemsetAsync(err_all.p, 0, 4 * sizeof(unsigned int), st));
  launch_pdl(k_box_reset, 1, 256, st, nbox, box.p); count_launch();
  {
    Scope sc(this, PH_INGEST);
    launch_pdl(k_ingest, grid(N), 256, st, N, bid.p, box.p, x.p, v.p, m.p, u.p, h.p, prm.gamma_kernel, H_in.p);
    count_launch();
  }
  const int box_bits = ceil_log2(nbox);
  const int dc = std::min(std::min(prm.max_depth, SPH_MAX_DEPTH), (64 - box_bits) / 3);
  launch_pdl(k_check_shape, 1, 256, st, nbox, box.p, dc, prm.split_headroom, err_all.p); count_launch();
  long long l0;
  int ev = prof_begin(PH_SORT, &l0);
  launch_pdl(k_keys, grid(N), 256, st, N, dcap, bid.p, box.p, x.p, key.p, perm.p); count_launch();
  radix_sort(key.p, perm.p, key_tmp.p, perm_tmp.p, N, key_bits, rs_scratch.p, st);
  launch_pdl(k_gather_sorted, grid(N), 256, st, N, perm.p, H_in.p, v.p, u.p, bid.p, box.p, a_in.p, vpred, Hs.p,
             vel4.p); count_launch();
  prof_end(PH_SORT, ev, l0);
  // the tree: a split that the depth bound blocks is flagged (capped)
  ev = prof_begin(PH_TREE, &l0);
  CKB(cudaMemsetAsync(t_n.p, 0, 8 * sizeof(int), st));
  CKB(cudaMemsetAsync(top_at.p, 0xff, N * sizeof(int), st));
  launch_pdl(k_top_nodes, grid(N), 256, st, N, dcap, box_shift, box.p, key.p, T, cap_nodes, top_at.p, err_all.p);
  count_launch();
  launch_pdl(k_frontier_init, 1, 1, st, T, cap_nodes); count_launch();
  const int rounds = dcap - kmin + 1;
  for (int r = 0; r < rounds; ++r) {
    launch_pdl(k_tree_round, nsm * 8, 256, st, T, box.p, Hs.p, key.p, dcap, prm.leaf_max, prm.split_frac,
               r + 1 < rounds ? 1 : 0, 1, cap_nodes, err_all.p); count_launch();
  }
  prof_end(PH_TREE, ev, l0);
  // the lists on st, the particle side on the side stream (as a build does)
  CKB(cudaEventRecord(ev_fork, st));
  CKB(cudaStreamWaitEvent(st_side, ev_fork, 0));
  ev = prof_begin(PH_LISTS, &l0);
  CKB(cudaMemsetAsync(l_counts.p, 0, 8 * sizeof(int), st));
  launch_pdl(k_items_top, grid(13ll * std::min<long long>(N, cap_nodes)), 256, st, cap_nodes, T, box.p, key.p,
             top_at.p, dcap, box_shift, Lq, cap_queue, err_all.p); count_launch();
  for (int r = 0; r < rounds; ++r) {
    const int in = r & 1;
    CKB(cudaMemsetAsync(l_counts.p + 2 + (in ^ 1), 0, sizeof(int), st));
    launch_pdl(k_items_expand, nsm * 8, 256, st, in, T, box.p, Lq, cap_queue, cap_self, cap_pair, err_all.p,
               prm.split_headroom); count_launch();
  }
  prof_end(PH_LISTS, ev, l0);
  cudaStream_t ss = st_side;
  ev = prof_begin(PH_SHIFT, &l0, ss);
  launch_pdl(k_leaves, nsm * 8, 256, ss, T, cap_nodes, leaf_of.p); count_launch();
  launch_pdl(k_leaf_partition, nsm * 8, 256, ss, T, cap_nodes, box.p, Hs.p, lsrc.p); count_launch();
  launch_pdl(k_apply_partition, grid(N), 256, ss, N, lsrc.p, perm.p, perm_tmp.p, key.p, key_tmp.p, Hs.p, Hs_tmp.p,
             vel4.p, vel4_tmp.p); count_launch();
  perm.swap(perm_tmp);
  key.swap(key_tmp);
  Hs.swap(Hs_tmp);
  vel4.swap(vel4_tmp);
  launch_pdl(k_shift, grid(N), 256, ss, N, box_shift, key.p, perm.p, leaf_of.p, T, box.p, x.p, m.p, Hs.p, pos4.p,
             cen4.p); count_launch();
  launch_pdl(k_tile_flags, nsm * 8, 256, ss, T, cap_nodes, box_shift, box.p, Hs.p, key.p, tflag.p, prm.cluster_max);
  count_launch();
  exclusive_scan(tflag.p, texcl.p, N, rs_scratch.p, reinterpret_cast<unsigned int*>(dev_counters.p + 4), ss);
  launch_pdl(k_tile_table, grid(N), 256, ss, N, T, leaf_of.p, tflag.p, texcl.p, pos4.p, tile_of.p, TL,
             prm.cluster_max); count_launch();
  launch_pdl(k_cell_tiles, grid(cap_nodes), 256, ss, T, cap_nodes, tile_of.p); count_launch();
  prof_end(PH_SHIFT, ev, l0, ss);
  CKB(cudaEventRecord(ev_join, ss));
  CKB(cudaStreamWaitEvent(st, ev_join, 0));
  launch_pdl(k_particle_limits, grid(N), 256, st, N, T, leaf_of.p, hlimp.p); count_launch();
  // the sorted projections
  ev = prof_begin(PH_AXIS_SORT, &l0);
  CKB(cudaMemsetAsync(big_count.p, 0, sizeof(unsigned long long), st));
  CKB(cudaMemsetAsync(mid_count.p, 0, sizeof(unsigned int), st));
  launch_pdl(k_mark_axes, nsm * 8, 256, st, Lq, cap_pair, T); count_launch();
  launch_pdl(k_sort_alloc, grid(cap_nodes), 256, st, T, cap_nodes, Lq, big_node.p, big_axis.p, big_off.p, big_count.p,
             cap_big, mid_seg.p, mid_count.p, (unsigned int)sort_r.n, (unsigned int)ckey.n, err_all.p);
  count_launch();
  launch_task_offsets(*this);
  launch_task_items(*this);
  if (prm.sort_merge)
    launch_pdl(k_sort_merge, nsm * 8, 256, st, mid_seg.p, mid_count.p, T, TL, sort_r.p, sort_i.p);
  else
    launch_pdl(k_sort_small, nsm * 8, 256, st, mid_seg.p, mid_count.p, T, TL, sort_r.p, sort_i.p);
  count_launch();
  // cells of many clusters: one global sort over the key storage, its unused
  // entries holding the largest key so that they sort last
  CKB(cudaMemsetAsync(ckey.p, 0xff, ckey.n * sizeof(unsigned long long), st));
  launch_pdl(k_sort_big_keys, nsm * 8, 256, st, -1, big_node.p, big_axis.p, big_off.p, T, TL, ckey.p, cval.p,
             big_count.p, cap_big); count_launch();
  radix_sort(ckey.p, cval.p, ckey_tmp.p, cval_tmp.p, (long long)ckey.n, 32 + ceil_log2((long long)cap_big + 1),
             rs_scratch.p, st);
  launch_pdl(k_sort_big_scatter, nsm * 8, 256, st, -1, big_node.p, big_axis.p, big_off.p, T, TL, cval.p, sort_r.p,
             sort_i.p, big_count.p, cap_big); count_launch();
  prof_end(PH_AXIS_SORT, ev, l0);
  CKB(cudaMemcpyAsync(x_build.p, x.p, 3 * N * sizeof(double), cudaMemcpyDeviceToDevice, st));
  return SPH_OK;
}

sph_status Engine::capture_build_graph() {
  drop_build_graph();
  // capacities with room to grow: a count past one makes the build not hold, and
  // the host completes that step with a build of its own
  const size_t cp = (size_t)(n_ptasks + n_ptasks / 4 + 1024), cs = (size_t)(n_stasks + n_stasks / 4 + 1024);
  CK(l_ptask.reserve(cp));
  CK(l_stask.reserve(cs));
  CK(l_plive.reserve(cp + cs));
  CK(g_live.reserve(l_plive.n));
  CK(l_nlive.reserve(1));
  Lq.p_task = l_ptask.p;
  Lq.s_task = l_stask.p;
  Lq.p_live = l_plive.p;
  Lq.n_live = l_nlive.p;
  CK(sort_r.reserve((size_t)(n_entries + n_entries / 4 + 4096)));
  CK(sort_i.reserve(sort_r.n));
  const size_t nb = (size_t)(n_big_entries + n_big_entries / 4 + 4096);
  CK(ckey.reserve(nb));
  CK(ckey_tmp.reserve(ckey.n));
  CK(cval.reserve(ckey.n));
  CK(cval_tmp.reserve(ckey.n));
  if (rs_scratch.n < (size_t)radix_scratch_words((long long)std::max<size_t>((size_t)N, ckey.n)))
    CK(rs_scratch.reserve((size_t)radix_scratch_words((long long)std::max<size_t>((size_t)N, ckey.n))));
  CK(mid_seg.reserve(13 * (size_t)cap_nodes));
  CK(mid_count.reserve(1));
  CK(big_count.reserve(1));
  CK(gstat.reserve(4));
  CK(it_dev.reserve(4));
  {
    sph_status s = ensure_side_stream();
    if (s != SPH_OK) return s;
    s = rec_prepare();
    if (s != SPH_OK) return s;
  }
  if (prof) {
    while (gev_pool.size() < 64) {
      cudaEvent_t e;
      CK(cudaEventCreate(&e));
      gev_pool.push_back(e);
    }
  }
  const long long c0 = launch_count();
  const cudaStreamCaptureMode mode = cudaStreamCaptureModeThreadLocal;
  CKB(cudaGraphCreate(&bstep_g, 0));
  cudaGraphConditionalHandle ok, iter, frc;
  CKB(cudaGraphConditionalHandleCreate(&ok, bstep_g, 0, cudaGraphCondAssignDefault));
  CKB(cudaGraphConditionalHandleCreate(&iter, bstep_g, 0, cudaGraphCondAssignDefault));
  CKB(cudaGraphConditionalHandleCreate(&frc, bstep_g, 0, cudaGraphCondAssignDefault));
  // kick, drift, build and its check
  cudaGraph_t g1 = nullptr;
  gcap = true;
  prof_into_graph = prof;
  CKB(cudaStreamBeginCapture(st, mode));
  // the force decision of this launch starts out false (the later force phases read it)
  CKB(cudaMemsetAsync(it_dev.p + 3, 0, sizeof(int), st));
  {
    Scope sc(this, PH_STEP);
    launch_kick(*this);
    launch_drift(*this);
  }
  {
    sph_status s = enqueue_captured_build();
    if (s != SPH_OK) return s;
  }
  launch_pdl(k_check_build, 1, 1, st, ok, err_all.p, t_n.p, cap_nodes, l_counts.p, cap_self, cap_pair, gb_last_q,
             (unsigned int)l_ptask.n, (unsigned int)l_stask.n, big_count.p, cap_big, gstat.p); count_launch();
  CKB(cudaStreamEndCapture(st, &g1));
  gb_build = launch_count() - c0;
  cudaGraphNode_t n1, n2, n3, n4;
  CKB(cudaGraphAddChildGraphNode(&n1, bstep_g, nullptr, 0, g1));
  cudaGraphDestroy(g1);
  // IF the build held: the h iteration set up
  cudaGraphNodeParams cp_ = {};
  cp_.type = cudaGraphNodeTypeConditional;
  cp_.conditional.handle = ok;
  cp_.conditional.type = cudaGraphCondTypeIf;
  cp_.conditional.size = 1;
  CKB(cudaGraphAddNode(&n2, bstep_g, &n1, nullptr, 1, &cp_));
  cudaGraph_t body = cp_.conditional.phGraph_out[0];
  long long c1 = launch_count();
  CKB(cudaStreamBeginCaptureToGraph(st, body, nullptr, nullptr, 0, mode));
  launch_bracket_reset(*this);
  launch_set_active(*this);
  CKB(cudaMemsetAsync(dev_counters.p, 0, 4 * sizeof(int), st));
  CKB(cudaMemsetAsync(err_all.p, 0, 4 * sizeof(unsigned int), st));
  rec_enqueue_reset();
  launch_iter_start(*this, iter);
  CKB(cudaStreamEndCapture(st, &body));
  gb_setup = launch_count() - c1;
  // WHILE iterating: one density pass and its h update (timed as a whole below)
  cudaGraphNode_t prev = n2;
  int ev_iter = -1;
  if (prof) {
    ev_iter = (int)(2 * gprof_recs.size());
    cudaGraphNode_t e0;
    CKB(cudaGraphAddEventRecordNode(&e0, bstep_g, &prev, 1, gev_pool[ev_iter]));
    prev = e0;
  }
  cp_ = {};
  cp_.type = cudaGraphNodeTypeConditional;
  cp_.conditional.handle = iter;
  cp_.conditional.type = cudaGraphCondTypeWhile;
  cp_.conditional.size = 1;
  CKB(cudaGraphAddNode(&n3, bstep_g, &prev, nullptr, 1, &cp_));
  body = cp_.conditional.phGraph_out[0];
  c1 = launch_count();
  const bool keep_prof = prof;
  prof = false;                      // no per-pass events inside the loop
  prof_into_graph = false;
  CKB(cudaStreamBeginCaptureToGraph(st, body, nullptr, nullptr, 0, mode));
  launch_zero_density(*this, false);
  launch_gather_prep(*this, it_dev.p);
  launch_live_tasks(*this, true, it_dev.p);
  launch_density(*this, it_dev.p);
  launch_density_gather(*this);
  launch_ghost(*this, 1, 0, it_dev.p);
  launch_iter_next(*this, iter, frc);
  launch_mark_active_cells(*this);
  CKB(cudaStreamEndCapture(st, &body));
  prof = keep_prof;
  prof_into_graph = prof;
  gb_iter = launch_count() - c1;
  prev = n3;
  if (prof) {
    cudaGraphNode_t e1;
    CKB(cudaGraphAddEventRecordNode(&e1, bstep_g, &prev, 1, gev_pool[ev_iter + 1]));
    prev = e1;
    gprof_recs.push_back(GProfRec{PH_DENSITY, ev_iter, gb_iter});
  }
  // IF finished without a rebuild: force pass and the closing kick.  Timed, the
  // phases take one conditional node each, so that event nodes of the top graph
  // sit between them (a conditional body holds no events); a handle belongs to
  // one node, so the later ones take the decision from the flag k_iter_next left
  // in it_dev[3], one kernel node each.
  c1 = launch_count();
  prof = false;
  prof_into_graph = false;
  int nphase = 0;
  auto phase_if = [&](int phase, auto&& enqueue) -> sph_status {
    cudaGraphConditionalHandle h = frc;
    if (nphase > 0) {
      CKB(cudaGraphConditionalHandleCreate(&h, bstep_g, 0, cudaGraphCondAssignDefault));
      cudaGraphNode_t ks;
      CKB(add_cond_set_node(&ks, bstep_g, &prev, 1, h, it_dev.p + 3));
      count_launches(1);
      prev = ks;
    }
    ++nphase;
    int ev = -1;
    if (keep_prof) {
      ev = (int)(2 * gprof_recs.size());
      cudaGraphNode_t e0;
      CKB(cudaGraphAddEventRecordNode(&e0, bstep_g, &prev, 1, gev_pool[ev]));
      prev = e0;
    }
    cudaGraphNodeParams q = {};
    q.type = cudaGraphNodeTypeConditional;
    q.conditional.handle = h;
    q.conditional.type = cudaGraphCondTypeIf;
    q.conditional.size = 1;
    cudaGraphNode_t nd;
    CKB(cudaGraphAddNode(&nd, bstep_g, &prev, nullptr, 1, &q));
    const long long l0 = launch_count();
    CKB(cudaStreamBeginCaptureToGraph(st, q.conditional.phGraph_out[0], nullptr, nullptr, 0, mode));
    enqueue();
    cudaGraph_t bg = nullptr;
    CKB(cudaStreamEndCapture(st, &bg));
    prev = nd;
    if (keep_prof) {
      cudaGraphNode_t e1;
      CKB(cudaGraphAddEventRecordNode(&e1, bstep_g, &prev, 1, gev_pool[ev + 1]));
      prev = e1;
      gprof_recs.push_back(GProfRec{phase, ev, launch_count() - l0});
    }
    return SPH_OK;
  };
  auto force_tasks = [&] {
    cudaMemsetAsync(facc.p, 0, N * sizeof(float4), st);
    cudaMemsetAsync(fvsig.p, 0, N * sizeof(float), st);
    launch_live_tasks(*this, false);
  };
  auto reduce = [&] {
    launch_reduce(*this);
    launch_save_acc(*this);
  };
  sph_status ps;
  if (keep_prof) {
    ps = phase_if(PH_FORCE_TASKS, force_tasks);
    if (ps == SPH_OK) ps = phase_if(PH_FORCE, [&] { launch_force(*this); });
    if (ps == SPH_OK) ps = phase_if(PH_REDUCE, reduce);
    if (ps == SPH_OK) ps = phase_if(PH_STEP, [&] { launch_kick(*this); });
  } else {
    ps = phase_if(PH_FORCE, [&] {
      force_tasks();
      launch_force(*this);
      reduce();
      launch_kick(*this);
    });
  }
  prof = keep_prof;
  if (ps != SPH_OK) {
    gcap = false;
    return ps;
  }
  gb_force = launch_count() - c1;
  gcap = false;
  prof_into_graph = false;
  CKB(cudaGraphInstantiate(&bstep_x, bstep_g, 0));
  count_launches(-(launch_count() - c0));     // capturing launches nothing
  bgraph_ready = true;
  bgraph_prof = prof;
  return SPH_OK;
}

sph_status Engine::build_step_graph() {
  if (!bgraph_ready || bgraph_prof != prof) {
    sph_status s = capture_build_graph();
    if (s != SPH_OK) return s;
  }
  CK(cudaGraphLaunch(bstep_x, st));
  unsigned int gs = 0, ea = 0;
  int itv[2] = {0, 0}, tn[8], lc[8];
  unsigned int ntl = 0;
  unsigned long long bcw = 0;
  CK(cudaMemcpyAsync(&gs, gstat.p, sizeof(gs), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(&ea, err_all.p, sizeof(ea), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(itv, it_dev.p, sizeof(itv), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(tn, t_n.p, sizeof(tn), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(lc, l_counts.p, sizeof(lc), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(&ntl, dev_counters.p + 4, sizeof(ntl), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(&bcw, big_count.p, sizeof(bcw), cudaMemcpyDeviceToHost, st));
  unsigned int rc = 0;
  if (R.pool) CK(cudaMemcpyAsync(&rc, rec_ctr.p, sizeof(rc), cudaMemcpyDeviceToHost, st));
  CK(sync_stream());
  const bool held = gs == 1u;
  if (R.pool && held) {
    rec_used = rc;
    rec_need = std::max<long long>(rec_need, rc);
    rec_unread = false;
  }
  const bool rebuild = !held || (ea & ERR_REBUILD) != 0u;
  count_launches(gb_build + (held ? gb_setup + (long long)itv[0] * gb_iter + (rebuild ? 0 : gb_force) : 0));
  if (held) {
    // this build's sizes, as a host build leaves them
    n_nodes = tn[0];
    n_top = tn[3];
    depth_used = tn[5];
    depth_hint = tn[5];
    depth_hint_leaf = prm.leaf_max;
    n_selfs = lc[0];
    n_pairs = lc[1];
    n_segments = lc[4];
    n_entries = (unsigned int)lc[5];
    n_ptasks = lc[6];
    n_stasks = lc[7];
    n_tiles = ntl;
    n_big = (int)(bcw >> 40);
    n_big_entries = (long long)(bcw & ((1ull << 40) - 1ull));
    built = true;
    reusable = true;
    ++n_builds;
    graph_ready = false;
  }
  if (rebuild) {
    // kick and drift are done: complete the step with a host-driven build
    sph_status s = build();
    if (s != SPH_OK) return s;
    return step_rest_after_build();
  }
  ++steps_graph;
  rec_valid = R.pool != nullptr;
  if (bgraph_prof) {
    for (const GProfRec& r : gprof_recs) {
      float t = 0.0f;
      CK(cudaEventElapsedTime(&t, gev_pool[r.ev], gev_pool[r.ev + 1]));
      gprof_ms[r.phase] += t;
      gprof_calls[r.phase] += 1;
      gprof_launches[r.phase] += r.launches;
    }
  }
  have_density = have_ghost = have_force = have_acc = true;
  last_iters = itv[0];
  last_rebuilds = 0;
  last_gathered = 0;
  first_active = itv[1];
  long long nu = 0;
  if (itv[0] >= prm.h_max_iter) {
    int cnt = 0;
    CK(cudaMemsetAsync(dev_counters.p + 1, 0, sizeof(int), st));
    launch_count_unconverged(*this, dev_counters.p + 1);
    CK(cudaMemcpyAsync(&cnt, dev_counters.p + 1, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(sync_stream());
    nu = cnt;
  }
  last_unconverged = nu;
  if (nu > 0) return fail(SPH_E_NOT_CONVERGED, std::to_string(nu) + " particles did not converge");
  return SPH_OK;
}

// After a host-driven build inside a step whose kick and drift are done: the h
// iteration, the force pass and the closing kick.
sph_status Engine::step_rest_after_build() {
  ++steps_host;
  sph_status hs = h_update(nullptr, nullptr);
  if (hs != SPH_OK && hs != SPH_E_NOT_CONVERGED) return hs;
  sph_status s = force();
  if (s != SPH_OK) return s;
  {
    Scope sc(this, PH_STEP);
    launch_kick(*this);
  }
  CK(cudaGetLastError());
  return hs;
}

// Leaf-size autotuning: time build + density + force for each candidate
// leaf_max (the split threshold of Section II-B; the paper uses 400 on its CPUs)
// and keep the fastest.
sph_status Engine::tune(int* best_out) {
  // leaf_max over its candidates with clusters of 32, then the cluster size at the
  // best leaf_max: times build + density + force (the mean of two repetitions
  // after one that warms up allocations)
  // (above the paper's 400: on GB300 larger leaves, fewer and heavier tasks, can pay)
  static const int cand[] = {24, 32, 48, 64, 96, 128, 192, 256, 400, 600, 800, 1200, 1600, 2400, 3200, 4800};
  static const int ccand[] = {16, 24};
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  const int keep = prm.leaf_max, keep_c = prm.cluster_max;
  tune_ms.clear();
  auto time_config = [&](int leaf, int cmax, float* ms_out) -> sph_status {
    prm.leaf_max = leaf;
    prm.cluster_max = cmax;
    float tot = 0.0f;
    for (int rep = 0; rep < 3; ++rep) {
      CK(cudaEventRecord(e0, st));
      sph_status s = build();
      if (s == SPH_OK) s = density();
      if (s == SPH_OK) s = force();
      if (s != SPH_OK) return s;
      CK(cudaEventRecord(e1, st));
      CK(cudaEventSynchronize(e1));
      float ms = 0.0f;
      CK(cudaEventElapsedTime(&ms, e0, e1));
      if (rep > 0) tot += ms;
    }
    *ms_out = tot / 2;
    return SPH_OK;
  };
  float best_ms = 1e30f;
  int best = keep, best_c = 32;
  sph_status s = SPH_OK;
  for (int c : cand) {
    float ms = 0.0f;
    s = time_config(c, 32, &ms);
    if (s != SPH_OK) break;
    tune_ms.push_back(std::make_pair(c, ms));
    if (ms < best_ms) {
      best_ms = ms;
      best = c;
    }
  }
  for (int cc : ccand) {
    if (s != SPH_OK) break;
    float ms = 0.0f;
    s = time_config(best, cc, &ms);
    if (s == SPH_OK && ms < best_ms) {
      best_ms = ms;
      best_c = cc;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s != SPH_OK) {
    prm.leaf_max = keep;
    prm.cluster_max = keep_c;
    return s;
  }
  prm.leaf_max = best;
  prm.cluster_max = best_c;
  built = have_density = have_ghost = have_force = false;
  reusable = false;
  if (best_out) *best_out = best;
  return SPH_OK;
}

sph_status Engine::cfl_dt(int b, double* dt) {
  if (!have_force) return fail(SPH_E_NOT_BUILT, "cfl_dt needs a force pass");
  const long long o = off[b], n = spec[b].n;
  std::vector<float> H(n), vs(n);
  CK(cudaMemcpyAsync(H.data(), Hs.p + o, n * sizeof(float), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(vs.data(), fvsig.p + o, n * sizeof(float), cudaMemcpyDeviceToHost, st));
  CK(sync_stream());
  double hmin = INFINITY, vmax = 0.0;
  for (long long p = 0; p < n; ++p) {
    hmin = std::min(hmin, (double)H[p]);
    vmax = std::max(vmax, (double)vs[p]);
  }
  *dt = vmax > 0 ? prm.c_cfl * hmin / vmax : INFINITY;
  return SPH_OK;
}

// ----------------------------------------------------------------------- outputs
sph_status Engine::get(int b, int field, void* dst, long long n, int mem) {
  sph_status s = get_async(b, field, dst, n, mem, staging.p);
  if (s == SPH_OK && mem != SPH_MEM_DEVICE) CK(sync_stream());
  return s;
}

// Several fields with one synchronisation: each field that is gathered goes
// through its own staging region.
sph_status Engine::get_fields(int b, int nf, const int* fields, void* const* dsts, const long long* ns, int mem) {
  if (nf < 0 || (nf > 0 && (!fields || !dsts || !ns))) return fail(SPH_E_INVALID, "null field list");
  size_t need = 0;
  for (int k = 0; k < nf; ++k) need += (size_t)std::max<long long>(ns[k], 0) * 3 * sizeof(double) / 2 + 256;
  CK(staging_many.reserve(need));
  size_t at = 0;
  for (int k = 0; k < nf; ++k) {
    sph_status s = get_async(b, fields[k], dsts[k], ns[k], mem, staging_many.p + at);
    if (s != SPH_OK) return s;
    at += (size_t)std::max<long long>(ns[k], 0) * 3 * sizeof(double) / 2 + 256;
  }
  if (mem != SPH_MEM_DEVICE) CK(sync_stream());
  return SPH_OK;
}

// One field, enqueued on the stream (host destinations complete at the next
// synchronisation); gathered fields pass through the staging region stg.
sph_status Engine::get_async(int b, int field, void* dst, long long n, int mem, unsigned char* stg) {
  if (b < 0 || b >= nbox) return fail(SPH_E_INVALID, "box index out of range");
  if (!dst) return fail(SPH_E_INVALID, "null destination");
  const long long o = off[b], nb = spec[b].n;
  const cudaMemcpyKind kind = mem == SPH_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (field == SPH_FIELD_REDUCTIONS) {
    if (n != 8) return fail(SPH_E_INVALID, "reductions need n = 8");
    if (!have_force) return fail(SPH_E_NOT_BUILT, "no force pass yet");
    CK(cudaMemcpyAsync(dst, red.p + 8 * b, 8 * sizeof(double), kind, st));
    return SPH_OK;
  }
  if (n != nb) return fail(SPH_E_INVALID, "n does not match the box's particle count");
  size_t bytes = 0;
  const void* src = nullptr;
  switch (field) {
    case SPH_FIELD_X: src = x.p + 3 * o; bytes = 3 * nb * sizeof(double); break;
    case SPH_FIELD_V: src = v.p + 3 * o; bytes = 3 * nb * sizeof(float); break;
    case SPH_FIELD_U: src = u.p + o; bytes = nb * sizeof(float); break;
    case SPH_FIELD_H: src = h.p + o; bytes = nb * sizeof(float); break;
    case SPH_FIELD_CONVERGED:
      if (!have_density) return fail(SPH_E_NOT_BUILT, "no density pass yet");
      src = conv.p + o; bytes = nb * sizeof(int); break;
    default: break;
  }
  if (src) {
    CK(cudaMemcpyAsync(dst, src, bytes, kind, st));
    return SPH_OK;
  }
  int per = 1;
  switch (field) {
    case SPH_FIELD_RHO: case SPH_FIELD_DRHO_DH: case SPH_FIELD_NW: case SPH_FIELD_NNGB: case SPH_FIELD_COUNT:
      if (!have_density) return fail(SPH_E_NOT_BUILT, "no density pass yet");
      break;
    case SPH_FIELD_P: case SPH_FIELD_C: case SPH_FIELD_F:
      if (!have_ghost) return fail(SPH_E_NOT_BUILT, "no ghost pass yet");
      break;
    case SPH_FIELD_A: per = 3;  // fallthrough
    case SPH_FIELD_DUDT: case SPH_FIELD_VSIG:
      if (!have_force) return fail(SPH_E_NOT_BUILT, "no force pass yet");
      break;
    case SPH_FIELD_FORCE_COUNT:
      if (!have_force || !have_fcount) return fail(SPH_E_NOT_BUILT, "no force pass with pair counting yet");
      break;
    default: return fail(SPH_E_INVALID, "unknown field");
  }
  void* out = mem == SPH_MEM_DEVICE ? dst : (void*)stg;
  {
    Scope sc(this, PH_OUTPUT);
    launch_get_field(*this, o, nb, field, out);
  }
  CK(cudaGetLastError());
  if (mem != SPH_MEM_DEVICE) CK(cudaMemcpyAsync(dst, stg, per * nb * 4, cudaMemcpyDeviceToHost, st));
  return SPH_OK;
}

sph_status Engine::set_field(int b, int field, const void* src, long long n, int mem) {
  if (b < 0 || b >= nbox) return fail(SPH_E_INVALID, "box index out of range");
  if (!src) return fail(SPH_E_INVALID, "null source");
  const long long o = off[b], nb = spec[b].n;
  if (n != nb) return fail(SPH_E_INVALID, "n does not match the box's particle count");
  if (field == SPH_FIELD_H) {
    const float* hsrc = static_cast<const float*>(src);
    if (mem != SPH_MEM_DEVICE) {
      CK(cudaMemcpyAsync(staging.p, src, nb * sizeof(float), cudaMemcpyHostToDevice, st));
      hsrc = reinterpret_cast<const float*>(staging.p);
    }
    launch_set_h(*this, b, hsrc);
    CK(cudaGetLastError());
    built = have_density = have_ghost = have_force = false;
    reusable = false;
    return SPH_OK;
  }
  if (field != SPH_FIELD_A && field != SPH_FIELD_DUDT) return fail(SPH_E_INVALID, "field cannot be set");
  const int per = field == SPH_FIELD_A ? 3 : 1;
  const float* dsrc = static_cast<const float*>(src);
  if (mem != SPH_MEM_DEVICE) {
    CK(cudaMemcpyAsync(staging.p, src, per * nb * sizeof(float), cudaMemcpyHostToDevice, st));
    dsrc = reinterpret_cast<const float*>(staging.p);
  }
  if (!have_acc) CK(cudaMemsetAsync(a_in.p + o, 0, nb * sizeof(float4), st));
  launch_set_acc(*this, o, nb, field == SPH_FIELD_A ? 0 : 1, dsrc);
  CK(cudaGetLastError());
  have_acc = true;
  return SPH_OK;
}

sph_status Engine::stats(int b, sph_stats* o) {
  std::memset(o, 0, sizeof(*o));
  o->n_particles = spec[b].n;
  o->n_cells = n_nodes;
  o->n_selfs = n_selfs;
  o->n_leaves = n_selfs;
  o->n_pairs = n_pairs;
  o->n_sort_segments = n_segments;
  o->n_sorted_entries = n_entries;
  o->top_level = hbox.empty() ? 0 : hbox[b].k;
  o->depth = depth_used;
  o->h_iterations = last_iters;
  o->rebuilds = last_rebuilds;
  o->builds = n_builds;
  o->reuses = n_reuses;
  o->h_active_after_first = first_active;
  o->h_gathered_passes = last_gathered;
  o->leaf_max = prm.leaf_max;
  o->cluster_max = prm.cluster_max;
  o->graph_steps = steps_graph;
  o->host_steps = steps_host;
  o->host_syncs = host_syncs;
  o->n_unconverged = last_unconverged;
  if (count_pairs) {
    unsigned long long c[16];
    CK(cudaMemcpyAsync(c, pc.p, sizeof(c), cudaMemcpyDeviceToHost, st));
    CK(sync_stream());
    o->density_pairs = (long long)(c[0] + c[3]);
    o->density_sides = (long long)(c[1] + c[4]);
    o->density_candidates = (long long)(c[2] + c[5]);
    o->density_pairs_cellpair = (long long)c[0];
    o->density_sides_cellpair = (long long)c[1];
    o->density_candidates_cellpair = (long long)c[2];
    o->force_pairs = (long long)(c[6] + c[8]);
    o->force_candidates = (long long)(c[7] + c[9]);
    o->force_pairs_cellpair = (long long)c[6];
    o->force_candidates_cellpair = (long long)c[7];
    o->guard_rechecks = (long long)c[10];
    o->force_tasks_replayed = (long long)c[11];
    o->force_tasks_culled = (long long)c[12];
  }
  return SPH_OK;
}

sph_status Engine::cells(int b, long long cap, int* level, int* ijk, int* count, int* split, long long* n_out) {
  if (!built) return fail(SPH_E_NOT_BUILT, "no decomposition built");
  std::vector<int> lv(n_nodes), bx(n_nodes), sp(n_nodes);
  std::vector<unsigned int> ct(n_nodes);
  std::vector<unsigned long long> ky(n_nodes);
  CK(cudaMemcpyAsync(lv.data(), t_level.p, n_nodes * sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(bx.data(), t_box.p, n_nodes * sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(sp.data(), t_split.p, n_nodes * sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(ct.data(), t_count.p, n_nodes * sizeof(unsigned int), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(ky.data(), t_key.p, n_nodes * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
  CK(sync_stream());
  long long k = 0;
  for (int id = 0; id < n_nodes; ++id) {
    if (bx[id] != b) continue;
    if (k < cap) {
      const int d = lv[id];
      const unsigned long long mort = d > 0 ? (ky[id] & ((1ull << (3 * d)) - 1ull)) : 0ull;
      if (level) level[k] = d;
      if (ijk) {
        ijk[3 * k] = (int)compact3(mort);
        ijk[3 * k + 1] = (int)compact3(mort >> 1);
        ijk[3 * k + 2] = (int)compact3(mort >> 2);
      }
      if (count) count[k] = (int)ct[id];
      if (split) split[k] = sp[id];
    }
    ++k;
  }
  *n_out = k;
  return SPH_OK;
}

sph_status Engine::interactions(int b, long long cap, int* kind, int* a, int* bb, int* axis, long long* n_out) {
  if (!built) return fail(SPH_E_NOT_BUILT, "no decomposition built");
  std::vector<int> bx(n_nodes), sa(n_selfs), pa(n_pairs), pb(n_pairs), pax(n_pairs);
  CK(cudaMemcpyAsync(bx.data(), t_box.p, n_nodes * sizeof(int), cudaMemcpyDeviceToHost, st));
  if (n_selfs) CK(cudaMemcpyAsync(sa.data(), l_self.p, n_selfs * sizeof(int), cudaMemcpyDeviceToHost, st));
  if (n_pairs) {
    CK(cudaMemcpyAsync(pa.data(), l_pa.p, n_pairs * sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(pb.data(), l_pb.p, n_pairs * sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(pax.data(), l_pax.p, n_pairs * sizeof(int), cudaMemcpyDeviceToHost, st));
  }
  CK(sync_stream());
  std::vector<int> local(n_nodes, -1);
  int c = 0;
  for (int id = 0; id < n_nodes; ++id)
    if (bx[id] == b) local[id] = c++;
  long long k = 0;
  auto put = [&](int kd, int x0, int x1, int ax) {
    if (k < cap) {
      if (kind) kind[k] = kd;
      if (a) a[k] = x0;
      if (bb) bb[k] = x1;
      if (axis) axis[k] = ax;
    }
    ++k;
  };
  for (int i = 0; i < n_selfs; ++i)
    if (bx[sa[i]] == b) put(0, local[sa[i]], -1, -1);
  for (int i = 0; i < n_pairs; ++i)
    if (bx[pa[i]] == b) put(1, local[pa[i]], local[pb[i]], pax[i]);
  *n_out = k;
  return SPH_OK;
}

}  // namespace sph

// =============================================================================== C-ABI
using sph::Engine;

struct sph_box {
  sph_ctx* ctx = nullptr;
  int device = 0;
  Engine* eng = nullptr;
};

static sph_status set_err(sph_ctx* c, sph_status s, const std::string& msg) {
  if (c) {
    std::lock_guard<std::mutex> g(c->mu);
    c->last = msg;
  }
  return s;
}

static sph_status from_engine(sph_box* b, sph_status s) {
  if (s != SPH_OK && b && b->ctx) set_err(b->ctx, s, b->eng->err);
  return s;
}

extern "C" {

void sph_params_default(sph_params* p) {
  if (!p) return;
  p->gamma_kernel = 1.825742f;
  p->n_ngb = 48.0f;
  p->gamma_gas = 5.0f / 3.0f;
  p->alpha_visc = 2.0f;
  p->c_cfl = 0.3f;
  p->h_tol = 1e-4f;
  p->h_max_iter = 30;
  p->leaf_max = 400;
  p->split_frac = 0.875f;
  p->max_depth = 20;
  p->split_headroom = 0.1f;
  p->reuse = 0;
  p->sort_merge = 0;
  p->cluster_max = 32;
  p->compensated = -1;
  p->precision = 0;
  p->graphs = 1;
  p->pair_cache = 0;
  p->h_gather = 1;
}

sph_status sph_ctx_create(const sph_params* params, int device, sph_ctx** out) {
  if (!out) return SPH_E_INVALID;
  *out = nullptr;
  sph_params p;
  sph_params_default(&p);
  if (params) p = *params;
  if (!(p.gamma_kernel > 0) || !(p.n_ngb > 0) || !(p.gamma_gas > 1) || p.h_max_iter < 1 || p.leaf_max < 1 ||
      !(p.split_frac >= 0 && p.split_frac <= 1) || p.max_depth < 1 || !(p.h_tol > 0) || !(p.alpha_visc >= 0) ||
      !(p.split_headroom >= 0 && p.split_headroom < 1) || p.cluster_max < 1 || p.cluster_max > 32 ||
      (p.precision != 0 && p.precision != 1) || (p.graphs != 0 && p.graphs != 1) ||
      (p.pair_cache != 0 && p.pair_cache != 1) || (p.h_gather != 0 && p.h_gather != 1))
    return SPH_E_INVALID;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return SPH_E_INVALID;
  if (cudaSetDevice(device) != cudaSuccess) return SPH_E_CUDA;
  sph_ctx* c = new sph_ctx;
  c->prm = p;
  c->device = device;
  if (cudaStreamCreateWithFlags(&c->own, cudaStreamNonBlocking) != cudaSuccess) {
    delete c;
    return SPH_E_CUDA;
  }
  c->cur = c->own;
  *out = c;
  return SPH_OK;
}

sph_status sph_ctx_set_stream(sph_ctx* c, void* stream) {
  if (!c) return SPH_E_INVALID;
  c->cur = stream ? (cudaStream_t)stream : c->own;
  return SPH_OK;
}

void* sph_ctx_stream(sph_ctx* c) { return c ? (void*)c->cur : nullptr; }

sph_status sph_ctx_destroy(sph_ctx* c) {
  if (!c) return SPH_E_INVALID;
  {
    std::lock_guard<std::mutex> g(c->mu);
    if (c->live > 0) {
      c->last = "context still has live boxes or servers";
      return SPH_E_BUSY;
    }
  }
  cudaSetDevice(c->device);
  if (c->own) cudaStreamDestroy(c->own);
  delete c;
  return SPH_OK;
}

const char* sph_last_error(sph_ctx* c) { return c ? c->last.c_str() : "null context"; }

sph_status sph_box_create(sph_ctx* c, int64_t n, double L, int periodic, sph_box** out) {
  if (!c || !out) return SPH_E_INVALID;
  *out = nullptr;
  if (n < 1 || n > (1ll << 31) - 1 || !(L > 0) || !std::isfinite(L))
    return set_err(c, SPH_E_INVALID, "box needs 1 <= n < 2^31 particles and a finite L > 0");
  cudaSetDevice(c->device);
  sph_box* b = new sph_box;
  b->ctx = c;
  b->device = c->device;
  b->eng = new Engine(c->prm, c->device, c->cur);
  sph_status s = b->eng->set_boxes({sph::BoxSpec{L, n, periodic ? 1 : 0}});
  if (s != SPH_OK) {
    set_err(c, s, b->eng->err);
    delete b->eng;
    delete b;
    return s == SPH_E_CUDA ? SPH_E_OOM : s;
  }
  {
    std::lock_guard<std::mutex> g(c->mu);
    c->live++;
  }
  *out = b;
  return SPH_OK;
}

#define BOX_PRE(b)                       \
  if (!(b) || !(b)->eng) return SPH_E_INVALID; \
  cudaSetDevice((b)->ctx->device);       \
  (b)->eng->st = (b)->ctx->cur;

sph_status sph_box_set(sph_box* b, const double* x, const float* v, const float* m, const float* u, const float* h,
                       int mem) {
  BOX_PRE(b);
  return from_engine(b, b->eng->set_particles(0, x, v, m, u, h, mem));
}

sph_status sph_box_set_field(sph_box* b, int field, const void* src, int64_t n, int mem) {
  BOX_PRE(b);
  return from_engine(b, b->eng->set_field(0, field, src, n, mem));
}

sph_status sph_box_set_owned(sph_box* b, int64_t n_owned) {
  BOX_PRE(b);
  if (n_owned < 0 || n_owned > b->eng->spec[0].n) return set_err(b->ctx, SPH_E_INVALID, "n_owned must be in 0..n");
  b->eng->hbox[0].nown = n_owned;
  b->eng->have_force = false;       // the sums of the last force pass counted other particles
  return from_engine(b, b->eng->upload_boxes());
}

sph_status sph_box_count_pairs(sph_box* b, int on) {
  BOX_PRE(b);
  b->eng->count_pairs = on != 0;
  return SPH_OK;
}

sph_status sph_box_destroy(sph_box* b) {
  if (!b) return SPH_E_INVALID;
  cudaSetDevice(b->device);
  cudaStreamSynchronize(b->eng->st);
  delete b->eng;
  {
    std::lock_guard<std::mutex> g(b->ctx->mu);
    b->ctx->live--;
  }
  delete b;
  return SPH_OK;
}

sph_status sph_build(sph_box* b) {
  BOX_PRE(b);
  return from_engine(b, b->eng->build());
}

sph_status sph_density(sph_box* b) {
  BOX_PRE(b);
  return from_engine(b, b->eng->density());
}

sph_status sph_h_update(sph_box* b, int64_t* n_unconverged, int32_t* iterations) {
  BOX_PRE(b);
  long long nu = 0;
  int it = 0;
  sph_status s = b->eng->h_update(&nu, &it);
  if (n_unconverged) *n_unconverged = nu;
  if (iterations) *iterations = it;
  return from_engine(b, s);
}

sph_status sph_force(sph_box* b) {
  BOX_PRE(b);
  return from_engine(b, b->eng->force());
}

sph_status sph_step(sph_box* b, double dt) {
  BOX_PRE(b);
  if (!(dt >= 0) || !std::isfinite(dt)) return set_err(b->ctx, SPH_E_INVALID, "dt must be finite and >= 0");
  return from_engine(b, b->eng->step(dt));
}

sph_status sph_cfl_dt(sph_box* b, double* dt) {
  BOX_PRE(b);
  if (!dt) return SPH_E_INVALID;
  return from_engine(b, b->eng->cfl_dt(0, dt));
}

sph_status sph_get(sph_box* b, int field, void* dst, int64_t n, int mem) {
  BOX_PRE(b);
  return from_engine(b, b->eng->get(0, field, dst, n, mem));
}

sph_status sph_get_fields(sph_box* b, int32_t n_fields, const int32_t* fields, void* const* dst, const int64_t* n,
                          int mem) {
  BOX_PRE(b);
  if (n_fields < 0 || n_fields > 64) return set_err(b->ctx, SPH_E_INVALID, "n_fields must be in 0..64");
  std::vector<int> f(fields ? fields : nullptr, fields ? fields + n_fields : nullptr);
  std::vector<long long> nn(n ? n : nullptr, n ? n + n_fields : nullptr);
  if (n_fields > 0 && (!fields || !n || !dst)) return set_err(b->ctx, SPH_E_INVALID, "null field list");
  return from_engine(b, b->eng->get_fields(0, n_fields, f.data(), dst, nn.data(), mem));
}

sph_status sph_box_profile(sph_box* b, int on) {
  BOX_PRE(b);
  b->eng->prof = on != 0;
  b->eng->prof_reset();
  return SPH_OK;
}

sph_status sph_get_profile(sph_box* b, int32_t cap, sph_profile_entry* out, int32_t* n_out) {
  BOX_PRE(b);
  if (!n_out) return SPH_E_INVALID;
  std::vector<double> ms;
  std::vector<long long> calls, launches;
  sph_status s = b->eng->prof_read(ms, calls, launches);
  if (s != SPH_OK) return from_engine(b, s);
  for (int k = 0; k < sph::PH_COUNT && k < cap; ++k) {
    std::memset(out[k].name, 0, sizeof(out[k].name));
    std::strncpy(out[k].name, sph::kPhaseNames[k], sizeof(out[k].name) - 1);
    out[k].calls = calls[k];
    out[k].launches = launches[k];
    out[k].ms = ms[k];
  }
  *n_out = sph::PH_COUNT;
  return SPH_OK;
}

int64_t sph_launch_count(void) { return sph::launch_count(); }

sph_status sph_measure_fp32_peak(sph_ctx* c, double* tflops) {
  if (!c || !tflops) return SPH_E_INVALID;
  if (cudaSetDevice(c->device) != cudaSuccess) return SPH_E_CUDA;
  int nsm = 0;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) return SPH_E_CUDA;
  float* scratch = nullptr;
  if (cudaMalloc(&scratch, (size_t)nsm * 8 * sizeof(float)) != cudaSuccess) return SPH_E_OOM;
  *tflops = sph::measure_fp32_peak(c->cur, nsm, scratch);
  const cudaError_t e = cudaGetLastError();
  cudaFree(scratch);
  return e == cudaSuccess ? SPH_OK : SPH_E_CUDA;
}

sph_status sph_box_tune(sph_box* b, int32_t* leaf_max) {
  BOX_PRE(b);
  int best = 0;
  sph_status s = b->eng->tune(&best);
  if (leaf_max) *leaf_max = best;
  return from_engine(b, s);
}

sph_status sph_box_set_cluster_max(sph_box* b, int32_t cluster_max) {
  BOX_PRE(b);
  if (cluster_max < 1 || cluster_max > 32) return set_err(b->ctx, SPH_E_INVALID, "cluster_max must be in 1..32");
  b->eng->prm.cluster_max = cluster_max;
  b->eng->built = b->eng->have_density = b->eng->have_ghost = b->eng->have_force = false;
  b->eng->reusable = false;
  return SPH_OK;
}

sph_status sph_box_set_leaf_max(sph_box* b, int32_t leaf_max) {
  BOX_PRE(b);
  if (leaf_max < 1) return set_err(b->ctx, SPH_E_INVALID, "leaf_max must be >= 1");
  b->eng->prm.leaf_max = leaf_max;
  b->eng->built = b->eng->have_density = b->eng->have_ghost = b->eng->have_force = false;
  return SPH_OK;
}

sph_status sph_get_stats(sph_box* b, sph_stats* out) {
  BOX_PRE(b);
  if (!out) return SPH_E_INVALID;
  return from_engine(b, b->eng->stats(0, out));
}

sph_status sph_get_cells(sph_box* b, int64_t cap, int32_t* level, int32_t* ijk, int32_t* count, int32_t* split,
                         int64_t* n_out) {
  BOX_PRE(b);
  if (!n_out) return SPH_E_INVALID;
  long long n = 0;
  sph_status s = b->eng->cells(0, cap, level, ijk, count, split, &n);
  *n_out = n;
  return from_engine(b, s);
}

sph_status sph_get_interactions(sph_box* b, int64_t cap, int32_t* kind, int32_t* a, int32_t* bb, int32_t* axis,
                                int64_t* n_out) {
  BOX_PRE(b);
  if (!n_out) return SPH_E_INVALID;
  long long n = 0;
  sph_status s = b->eng->interactions(0, cap, kind, a, bb, axis, &n);
  *n_out = n;
  return from_engine(b, s);
}

}  // extern "C"
