// Host-side engine of the GB300 SPH path: device buffers of a batch of boxes
// and the launch sequences of the build and the passes.  One engine drives one
// box (the C-ABI sph_box) or many boxes at once (the server).
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "sph.h"
#include "sph_internal.cuh"

namespace sph {

// A device array that only grows.
template <class T>
struct DBuf {
  T* p = nullptr;
  size_t n = 0;
  cudaError_t reserve(size_t want) {
    if (want <= n && p) return cudaSuccess;
    release();
    if (want == 0) want = 1;
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&p), want * sizeof(T));
    if (e != cudaSuccess) {
      p = nullptr;
      n = 0;
      return e;
    }
    n = want;
    return cudaSuccess;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
  }
  size_t bytes() const { return n * sizeof(T); }
  void swap(DBuf& o) {
    std::swap(p, o.p);
    std::swap(n, o.n);
  }
  ~DBuf() { release(); }
};

struct BoxSpec {
  double L;
  long long n;
  int periodic;
};

// Process-wide count of kernel launches made by the library (host side).
void count_launch();
long long launch_count();

// Phases of the path timed with CUDA events when profiling is on.
enum Phase {
  PH_INGEST, PH_SORT, PH_TREE, PH_LISTS, PH_SHIFT, PH_AXIS_SORT, PH_DENSITY, PH_DENSITY_TASKS, PH_GHOST,
  PH_FORCE, PH_FORCE_TASKS, PH_REDUCE, PH_STEP, PH_OUTPUT, PH_REUSE, PH_COUNT
};
extern const char* const kPhaseNames[PH_COUNT];

// Kernels and helpers implemented in build.cu / interact.cu.
void exclusive_scan(const unsigned int* in, unsigned int* out, long long n, unsigned int* tile_sums,
                    unsigned int* total, cudaStream_t st, const unsigned int* n_dev = nullptr,
                    const int* gate = nullptr);
long long radix_scratch_words(long long n);
void radix_sort(unsigned long long* k0, unsigned int* v0, unsigned long long* k1, unsigned int* v1, long long n,
                int bits, unsigned int* scratch, cudaStream_t st);

class Engine {
 public:
  Engine(const sph_params& prm, int device, cudaStream_t st);
  ~Engine();

  // ---- configuration -------------------------------------------------------
  sph_status set_boxes(const std::vector<BoxSpec>& boxes);   // (re)size for these boxes
  // New box layout where box b takes over the input-order state (x, v, m, u, h,
  // saved accelerations) of current box src[b], or starts empty (src[b] < 0)
  // for set_particles to fill; the moves run on the device.
  sph_status relayout(const std::vector<BoxSpec>& boxes, const std::vector<int>& src);
  // copy particle state of box b (host or device pointers)
  sph_status set_particles(int b, const double* x, const float* v, const float* m, const float* u, const float* h,
                           int mem);

  // ---- the hot path -----------------------------------------------------------
  sph_status build();
  sph_status reuse_or_build();        // keep the last decomposition while valid (prm.reuse), else build
  sph_status step_graph();            // a kept-decomposition step as one CUDA graph (prm.reuse)
  sph_status capture_step_graph();
  void drop_step_graph();
  sph_status build_step_graph();      // a step that rebuilds the decomposition, as one CUDA graph
  sph_status capture_build_graph();
  void drop_build_graph();
  sph_status enqueue_captured_build();
  sph_status step_host(bool moving);  // the rest of a step after its kick and drift, host-sequenced
  sph_status step_rest_after_build();
  sph_status density();                                        // one pass at the current h, all particles
  sph_status h_update(long long* n_unconverged, int* iterations);
  sph_status force();
  sph_status step(double dt);          // every box with the same dt
  sph_status step_boxes();             // every box with its own hbox[b].dt
  sph_status step_boxes_once();
  sph_status cfl_dt(int b, double* dt);
  sph_status tune(int* best_leaf_max);
  std::vector<std::pair<int, float>> tune_ms;   // (leaf_max, ms) of the last tune()
  sph_status get(int b, int field, void* dst, long long n, int mem);
  sph_status get_async(int b, int field, void* dst, long long n, int mem, unsigned char* stg);
  sph_status get_fields(int b, int nf, const int* fields, void* const* dsts, const long long* ns, int mem);
  sph_status set_field(int b, int field, const void* src, long long n, int mem);
  sph_status stats(int b, sph_stats* out);
  sph_status cells(int b, long long cap, int* level, int* ijk, int* count, int* split, long long* n_out);
  sph_status interactions(int b, long long cap, int* kind, int* a, int* bb, int* axis, long long* n_out);

  // ---- state -----------------------------------------------------------------
  sph_params prm;
  int device = 0;
  cudaStream_t st = nullptr;
  // Side stream of the build: after the tree, the particle-side kernels run on it
  // while the interaction lists are built on st (fork and join by events).
  // Created with the first build.
  cudaStream_t st_side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  int nsm = 148;
  std::string err;
  bool count_pairs = false;
  size_t footprint_bytes() const;

  std::vector<BoxSpec> spec;
  std::vector<long long> off;   // first particle of each box
  long long N = 0;
  int nbox = 0;
  std::vector<BoxDesc> hbox;
  int dcap = 0, box_shift = 0, kmin = 0, kmax = 0, key_bits = 0;

  // box table and input-order particle state (owned by the engine)
  DBuf<BoxDesc> box;
  DBuf<int> bid;
  DBuf<double> x;
  DBuf<float> v, m, u, h;
  DBuf<float4> hhist;             // roots of N~(h) = N_ngb of this step (x) and the three before (y, z, w), input order
  DBuf<int> hlev, hlev_old;       // per box: earlier roots held in hhist (0..3)
  DBuf<long long> hlev_src;       // relayout: source box of every new box (-1: new)
  DBuf<float> H_in, hlo, hhi;
  DBuf<int> conv;                 // 1 when h converged (input order)
  DBuf<float4> a_in;              // a and du/dt of the last force pass (input order)
  DBuf<long long> boff;           // first particle of each box, and N (device copy of off)
  // relayout targets
  DBuf<double> rl_x;
  DBuf<float> rl_v, rl_m, rl_u, rl_h;
  DBuf<float4> rl_hh;
  DBuf<float4> rl_a;
  DBuf<long long> rl_tab;

  // key-sorted particle state
  DBuf<unsigned long long> key, key_tmp;
  DBuf<unsigned int> perm, perm_tmp, rs_scratch;
  DBuf<float> Hs, hlimp;
  DBuf<float4> pos4, cen4, vel4;
  DBuf<unsigned int> leaf_of;
  DBuf<int> top_at;
  DBuf<unsigned char> act;        // still iterating h (sorted order)
  DBuf<float> Hs_tmp;
  DBuf<float4> vel4_tmp;
  DBuf<unsigned int> lsrc, tflag, texcl, tile_of;

  // clusters (capacity N)
  DBuf<unsigned int> tl_start, tl_n, tl_leaf;
  DBuf<float4> tl_lo, tl_hi, tl_cen;
  DBuf<unsigned char> tl_active, tl_changed;
  Tiles TL{};
  long long n_tiles = 0;

  // cell tree
  int cap_nodes = 0;
  DBuf<unsigned int> t_start, t_count, t_nsmall, t_axes, t_sortbase;
  DBuf<unsigned long long> t_key;
  DBuf<int> t_level, t_box, t_child, t_nchild, t_parent, t_split, t_n;
  DBuf<float> t_hmax;
  DBuf<double> t_hlim;
  DBuf<float4> t_cen;
  DBuf<unsigned char> t_active, t_changed;
  DBuf<unsigned int> t_alo, t_ahi, t_clo, t_chi;
  DBuf<uint4> mid_seg;            // (cell, axis, storage offset, clusters) of every shared-memory sort
  DBuf<unsigned int> mid_count;
  DBuf<unsigned int> t_tile0, t_ntile;
  Tree T{};

  // interaction lists
  int cap_self = 0, cap_pair = 0, cap_queue = 0;
  DBuf<int> l_self, l_pa, l_pb, l_pax, l_counts;
  DBuf<unsigned int> l_ptoff, l_stoff, scan_tmp, l_ptask, l_stask, l_nlive;
  DBuf<uint2> l_plive;
  // gathered later passes of the h iteration: per cluster the particles still
  // iterating (scanned to ranks), per leaf start its packed clusters (scanned to
  // their first index), the packed clusters (indices by rank, first rank and leaf
  // start, size), scan scratch and totals, the gathered tasks, their count and the
  // pass's choice
  DBuf<unsigned int> pk_cnt, pk_v, pk_idx, pk_sums, pk_tot, g_n;
  DBuf<uint2> pk_info, g_live;
  DBuf<unsigned char> pk_n;
  DBuf<int> gflag;
  long long n_ptasks = 0, n_stasks = 0;
  int partial_pass = 0;           // 1 while the density passes cover only particles still iterating h
  DBuf<int> q_kind[2], q_a[2], q_b[2], q_ax[2];
  Lists Lq{};

  // the pairs of the first density pass of an h iteration, kept for the force pass
  // (params.pair_cache): pool of batches in chunks, chunk links, chunk counter,
  // per-task records
  DBuf<unsigned int> rec_pool, rec_next, rec_ctr;
  DBuf<uint2> rec_pt, rec_st;
  PairRec R{};
  bool rec_valid = false;         // the records hold for the next force pass
  long long rec_need = 0;         // chunks the last recordings took (the pool grows to this)
  long long rec_used = 0;         // chunks the last recording read back took
  bool rec_unread = false;        // the last recording's chunk count was not read back yet
  sph_status rec_prepare();       // pool and record arrays sized for the next recording
  void rec_enqueue_reset();       // a recording starts with the next full density pass
  PairRec rec_for_force() const { return rec_valid ? R : PairRec{}; }

  // sorted projections
  DBuf<float> sort_r;
  DBuf<unsigned int> sort_i;
  int cap_big = 0;
  DBuf<int> big_node, big_axis;
  DBuf<unsigned long long> big_count;   // segments << 40 | entries
  DBuf<unsigned int> big_off;
  DBuf<unsigned long long> ckey, ckey_tmp;
  DBuf<unsigned int> cval, cval_tmp;

  // pass results (sorted order)
  DBuf<float4> dacc;              // sum m w, sum m q w', sum w, sum q w'
  DBuf<unsigned int> dcnt;
  DBuf<float4> ghost4;            // rho, f P / rho^2, c, f
  DBuf<float4> facc;              // a (3), du/dt
  DBuf<float> fvsig;
  DBuf<unsigned int> fcnt;        // force partners per particle (filled while counting pairs)
  DBuf<double> red;               // 8 per box
  DBuf<unsigned int> err_all;     // global error bits
  DBuf<unsigned long long> pc;    // pair counters per kernel (see commit_counters)
  DBuf<unsigned int> task_ctr;    // task counters of the four interaction kernels
  DBuf<int> dev_counters;         // [0] particles still active after a ghost pass
  DBuf<unsigned char> staging;    // output staging (input order)
  DBuf<unsigned char> staging_many;   // one region per field of a multi-field read

  // host mirrors of counts after the last build
  int n_nodes = 0, n_top = 0, n_selfs = 0, n_pairs = 0, n_segments = 0, n_big = 0;
  int depth_used = 0;       // deepest level holding a cell in the last build
  int depth_hint = 0;       // the depth bound of the next build is this plus one (0: none)
  int depth_hint_leaf = 0;  // the leaf size the hint was taken with
  long long n_entries = 0, n_big_entries = 0;
  int last_iters = 0, last_rebuilds = 0;
  long long first_active = 0;     // particles still iterating after the first density pass
  long long last_gathered = 0;    // later passes of the last host-driven h iteration that gathered
  int vpred = 0;                  // 1 inside a step after its drift: passes see v, u predicted to the step's end
  long long n_builds = 0, n_reuses = 0;
  bool reusable = false;          // the last full build can be kept (positions since then tracked)
  DBuf<double> x_build;           // positions at the last full build (input order)
  DBuf<unsigned long long> dmax_bits;   // per box: largest displacement since the build (double bits)
  DBuf<unsigned int> reuse_flag;
  DBuf<int> it_dev;               // captured step: iteration number, and the last iteration's active count
  // the captured step (valid for one decomposition)
  cudaGraph_t step_g = nullptr;
  cudaGraphExec_t step_x = nullptr;
  bool graph_ready = false, graph_off = false;
  long long g_pre = 0, g_keep = 0, g_iter = 0, g_force = 0;   // kernels per part
  // the captured rebuild step (valid while the boxes keep their top levels and the
  // capacities hold; a host build drops it, the next step captures it again)
  bool gcap = false;              // launches being captured for it: capacity-sized, counts on the device
  cudaGraph_t bstep_g = nullptr;
  cudaGraphExec_t bstep_x = nullptr;
  bool bgraph_ready = false, bgraph_prof = false;
  long long gb_build = 0, gb_setup = 0, gb_iter = 0, gb_force = 0;   // kernels per part
  int gb_last_q = 0;              // the expansion queue the last list round leaves empty
  DBuf<unsigned int> gstat;       // [0] 1 when the captured build held
  struct GProfRec {
    int phase, ev;
    long long launches;
  };
  std::vector<GProfRec> gprof_recs;   // phase events recorded inside the captured rebuild step
  std::vector<cudaEvent_t> gev_pool;
  std::vector<double> gprof_ms;
  std::vector<long long> gprof_calls, gprof_launches;
  bool prof_into_graph = false;
  long long steps_host = 0, steps_graph = 0, host_syncs = 0;
  long long steps_in_layout = 0;  // steps since the boxes were last laid out (a capture pays off after a few)
  long long last_unconverged = 0;
  bool built = false, have_density = false, have_ghost = false, have_force = false, have_acc = false;
  bool have_fcount = false;       // the last force pass counted pairs (fcnt is filled)

  // profiling: CUDA events around each phase on the engine's stream
  struct ProfRec {
    int phase, ev;
    long long launches;
  };
  bool prof = false;
  std::vector<ProfRec> prof_recs;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  int prof_begin(int phase, long long* l0, cudaStream_t on = nullptr);    // on: st when null
  void prof_end(int phase, int ev, long long l0, cudaStream_t on = nullptr);
  void prof_reset();
  sph_status prof_read(std::vector<double>& ms, std::vector<long long>& calls, std::vector<long long>& launches);
  struct Scope {
    Engine* e;
    int phase, ev;
    long long l0;
    Scope(Engine* en, int ph) : e(en), phase(ph), ev(-1), l0(0) { ev = e->prof_begin(ph, &l0); }
    ~Scope() { e->prof_end(phase, ev, l0); }
  };

  // helpers
  int grid(long long work, int threads = 256) const;
  cudaError_t sync_stream();
  sph_status cuda_fail(cudaError_t e, const char* where);
  sph_status fail(sph_status s, const std::string& msg);
  sph_status ensure_particle_capacity();
  sph_status ensure_side_stream();
  sph_status ensure_tree_capacity(int nodes);
  sph_status ensure_list_capacity(int selfs, int pairs, int queue);
  sph_status build_once(bool* retry);
  sph_status set_all_active();
  sph_status density_pass();
  sph_status ghost_pass(int mode, int it, int* n_active, bool* rebuild);
  sph_status upload_boxes();
};

}  // namespace sph

// C-ABI context: device, parameters, the stream every call launches on.
struct sph_ctx {
  sph_params prm;
  int device = 0;
  cudaStream_t own = nullptr;
  cudaStream_t cur = nullptr;
  std::string last;
  std::mutex mu;
  int live = 0;   // boxes and servers created on this context and not yet destroyed
};
