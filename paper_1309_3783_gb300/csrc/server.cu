// Batched, served boxes: a request queue in front of one engine that holds every
// admitted box on the device and advances all of them by one step per tick with
// a single batched pipeline (one launch per kernel for all boxes: the key sort,
// tree, interaction lists, axis sorts and the density/force kernels all run over
// the concatenated boxes; interactions never cross boxes).
//
// Admission is by device footprint against a byte budget, by a box count limit
// and by a bound on the particles one tick steps; waiting requests are admitted
// in submission order as finished boxes retire (continuous batching).  The boxes
// admitted in a tick first go through an intake pass on an engine of their own:
// the h iteration from their initial h and their starting forces, all new boxes
// batched.  They then join the resident boxes, moved device to device, and take
// their first kick-drift-kick step in the same tick, so that the batched step
// never carries the longer start-up iteration of a new box.  When the resident
// set changes, the boxes that stay keep their state on the device: the engine
// moves it to the new layout with one kernel.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <deque>
#include <map>
#include <string>
#include <vector>

#include "sph_engine.h"

namespace {

constexpr int kFields = 17;

struct Request {
  long long id = 0;
  double L = 1.0;
  int periodic = 1;
  long long n = 0;
  std::vector<double> x;
  std::vector<float> v, m, u, h;
  int n_steps = 0, done_steps = 0;
  double dt = 0.0;
  bool started = false;
  int state = 0;            // 0 waiting, 1 resident, 2 finished
  std::vector<float> step_ms;
  float intake_ms = -1.0f;  // device time of the intake pass it went through (-1: none)
  int intake_box = -1;      // its box in the intake engine during its admission tick
  std::vector<std::vector<unsigned char>> result;   // per field, caller order
};

size_t field_bytes(int f, long long n) {
  switch (f) {
    case SPH_FIELD_X: return 3 * n * sizeof(double);
    case SPH_FIELD_V: case SPH_FIELD_A: return 3 * n * sizeof(float);
    case SPH_FIELD_REDUCTIONS: return 8 * sizeof(double);
    default: return n * 4;
  }
}

}  // namespace

struct sph_server {
  sph_ctx* ctx = nullptr;
  int device = 0;
  cudaStream_t st = nullptr;
  sph::Engine* eng = nullptr;
  sph::Engine* intake = nullptr;   // start-up passes of the boxes admitted in a tick
  long long budget = 0;
  long long tick_budget = 0;       // particles a tick may step (0: no bound)
  int max_boxes = 0;
  long long next_id = 1;
  std::map<long long, Request> reqs;
  std::deque<long long> waiting;
  std::vector<long long> resident;
  std::vector<long long> layout;   // the boxes in the engine, in its order
  cudaEvent_t e0 = nullptr, e1 = nullptr, i0 = nullptr, i1 = nullptr;
  unsigned char* pin = nullptr;    // page-locked staging for the results of finished boxes
  size_t pin_cap = 0;
  std::string err;
};

static const long long kBytesPerParticle = 520;

static sph_status srv_fail(sph_server* s, sph_status st, const std::string& m) {
  s->err = m;
  return st;
}

// Bring the engine's box layout to the resident set: boxes that stay move on
// the device, new boxes are copied from their requests.
static sph_status apply_layout(sph_server* s) {
  sph::Engine& E = *s->eng;
  std::vector<sph::BoxSpec> spec;
  std::vector<int> src;
  for (long long id : s->resident) {
    const Request& r = s->reqs[id];
    spec.push_back(sph::BoxSpec{r.L, r.n, r.periodic});
    int from = -1;
    for (size_t k = 0; k < s->layout.size(); ++k)
      if (s->layout[k] == id) from = (int)k;
    src.push_back(from);
  }
  sph_status st = E.relayout(spec, src);
  if (st != SPH_OK) return srv_fail(s, st, E.err);
  for (size_t b = 0; b < s->resident.size(); ++b) {
    if (src[b] >= 0) continue;
    Request& r = s->reqs[s->resident[b]];
    if (r.intake_box >= 0) {
      // from the intake engine: converged h and starting forces, device to device
      sph::Engine& I = *s->intake;
      const long long o = I.off[r.intake_box];
      st = E.set_particles((int)b, I.x.p + 3 * o, I.v.p + 3 * o, I.m.p + o, I.u.p + o, I.h.p + o, SPH_MEM_DEVICE);
      if (st != SPH_OK) return srv_fail(s, st, E.err);
      cudaMemcpyAsync(E.a_in.p + E.off[b], I.a_in.p + o, r.n * sizeof(float4), cudaMemcpyDeviceToDevice, s->st);
      r.intake_box = -1;
      continue;
    }
    st = E.set_particles((int)b, r.x.data(), r.v.data(), r.m.data(), r.u.data(), r.h.data(), SPH_MEM_HOST);
    if (st != SPH_OK) return srv_fail(s, st, E.err);
    cudaMemsetAsync(E.a_in.p + E.off[b], 0, r.n * sizeof(float4), s->st);
  }
  // starting forces of new boxes come from their first (dt = 0) tick; the kick of
  // every box reads a_in, so the engine never recomputes forces on its own
  E.have_acc = true;
  s->layout = s->resident;
  return SPH_OK;
}

// The intake pass of the boxes admitted in this tick (requests with steps to
// run): one engine over all of them, built, h iterated from their initial h,
// forces computed; the boxes then join the resident layout from its buffers.
static sph_status run_intake(sph_server* s, const std::vector<long long>& ids) {
  if (ids.empty()) return SPH_OK;
  if (!s->intake) s->intake = new sph::Engine(s->ctx->prm, s->device, s->st);
  sph::Engine& I = *s->intake;
  I.st = s->st;
  std::vector<sph::BoxSpec> spec;
  for (long long id : ids) {
    const Request& r = s->reqs[id];
    spec.push_back(sph::BoxSpec{r.L, r.n, r.periodic});
  }
  sph_status st = I.set_boxes(spec);
  if (st != SPH_OK) return srv_fail(s, st, I.err);
  for (size_t k = 0; k < ids.size(); ++k) {
    Request& r = s->reqs[ids[k]];
    st = I.set_particles((int)k, r.x.data(), r.v.data(), r.m.data(), r.u.data(), r.h.data(), SPH_MEM_HOST);
    if (st != SPH_OK) return srv_fail(s, st, I.err);
  }
  cudaEventRecord(s->i0, s->st);
  st = I.build();
  if (st == SPH_OK) {
    st = I.h_update(nullptr, nullptr);
    if (st == SPH_E_NOT_CONVERGED) st = SPH_OK;
  }
  if (st == SPH_OK) st = I.force();
  cudaEventRecord(s->i1, s->st);
  if (st != SPH_OK) return srv_fail(s, st, I.err);
  cudaEventSynchronize(s->i1);
  float ms = 0.0f;
  cudaEventElapsedTime(&ms, s->i0, s->i1);
  for (size_t k = 0; k < ids.size(); ++k) {
    Request& r = s->reqs[ids[k]];
    r.intake_box = (int)k;
    r.intake_ms = ms;
    r.started = true;       // its first step runs in this tick
  }
  return SPH_OK;
}

static sph_status finish(sph_server* s, size_t b) {
  sph::Engine& E = *s->eng;
  Request& r = s->reqs[s->resident[b]];
  r.result.assign(kFields, {});
  for (int f = 0; f < kFields; ++f) {
    const long long n = f == SPH_FIELD_REDUCTIONS ? 8 : r.n;
    r.result[f].resize(field_bytes(f, r.n));
    sph_status st = E.get((int)b, f, r.result[f].data(), n, SPH_MEM_HOST);
    if (st != SPH_OK) r.result[f].clear();
  }
  r.state = 2;
  return SPH_OK;
}

static size_t round256(size_t v) { return (v + 255) & ~(size_t)255; }

// The results of several finished boxes: every field of every box is queued into
// page-locked staging and read with one synchronisation per chunk of at most
// kPinMax bytes, then copied to the requests.  Without page-locked memory the
// boxes go one field at a time.
static const size_t kPinMax = 256u << 20;

static sph_status finish_many(sph_server* s, const std::vector<size_t>& boxes) {
  sph::Engine& E = *s->eng;
  size_t i = 0;
  while (i < boxes.size()) {
    size_t j = i, bytes = 0;
    while (j < boxes.size()) {
      const Request& r = s->reqs[s->resident[boxes[j]]];
      size_t bb = 0;
      for (int f = 0; f < kFields; ++f) bb += round256(field_bytes(f, r.n));
      if (j > i && bytes + bb > kPinMax) break;
      bytes += bb;
      ++j;
    }
    if (bytes > s->pin_cap) {
      if (s->pin) cudaFreeHost(s->pin);
      s->pin = nullptr;
      s->pin_cap = 0;
      const size_t cap = std::max(bytes, std::min(2 * bytes, kPinMax));
      if (cudaMallocHost(reinterpret_cast<void**>(&s->pin), cap) != cudaSuccess) {
        cudaGetLastError();
        s->pin = nullptr;
        for (size_t k = i; k < j; ++k) finish(s, boxes[k]);
        i = j;
        continue;
      }
      s->pin_cap = cap;
    }
    std::vector<std::pair<size_t, bool>> at((j - i) * kFields);
    size_t off = 0;
    for (size_t k = i; k < j; ++k) {
      const Request& r = s->reqs[s->resident[boxes[k]]];
      for (int f = 0; f < kFields; ++f) {
        const long long n = f == SPH_FIELD_REDUCTIONS ? 8 : r.n;
        const sph_status st = E.get_async((int)boxes[k], f, s->pin + off, n, SPH_MEM_HOST, E.staging.p);
        at[(k - i) * kFields + f] = std::make_pair(off, st == SPH_OK);
        off += round256(field_bytes(f, r.n));
      }
    }
    if (cudaStreamSynchronize(s->st) != cudaSuccess) return srv_fail(s, SPH_E_CUDA, "reading results");
    for (size_t k = i; k < j; ++k) {
      Request& r = s->reqs[s->resident[boxes[k]]];
      r.result.assign(kFields, {});
      for (int f = 0; f < kFields; ++f) {
        const auto& a = at[(k - i) * kFields + f];
        if (a.second) r.result[f].assign(s->pin + a.first, s->pin + a.first + field_bytes(f, r.n));
      }
      r.state = 2;
    }
    i = j;
  }
  return SPH_OK;
}

extern "C" {

sph_status sph_server_create(sph_ctx* ctx, int64_t budget_bytes, int32_t max_boxes, sph_server** out) {
  if (!ctx || !out) return SPH_E_INVALID;
  *out = nullptr;
  const sph_ctx* cv = ctx;
  cudaSetDevice(cv->device);
  sph_server* s = new sph_server;
  s->ctx = ctx;
  s->device = cv->device;
  s->st = cv->cur;
  s->max_boxes = max_boxes > 0 ? max_boxes : 1 << 16;
  if (budget_bytes <= 0) {
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    budget_bytes = (int64_t)(0.8 * (double)fr);
  }
  s->budget = budget_bytes;
  s->eng = new sph::Engine(cv->prm, cv->device, s->st);
  cudaEventCreate(&s->e0);
  cudaEventCreate(&s->e1);
  cudaEventCreate(&s->i0);
  cudaEventCreate(&s->i1);
  {
    std::lock_guard<std::mutex> g(ctx->mu);
    ctx->live++;
  }
  *out = s;
  return SPH_OK;
}

sph_status sph_server_submit(sph_server* s, int64_t n, double L, int periodic, const double* x, const float* v,
                             const float* m, const float* u, const float* h, int32_t n_steps, double dt, int64_t* id) {
  if (!s || !id || !x || !v || !m || !u || !h) return SPH_E_INVALID;
  if (n < 1 || !(L > 0) || n_steps < 0 || !(dt >= 0)) return srv_fail(s, SPH_E_INVALID, "bad request");
  if ((long long)n * kBytesPerParticle > s->budget) return srv_fail(s, SPH_E_OOM, "box can never fit the budget");
  Request r;
  r.id = s->next_id++;
  r.L = L;
  r.periodic = periodic ? 1 : 0;
  r.n = n;
  r.x.assign(x, x + 3 * n);
  r.v.assign(v, v + 3 * n);
  r.m.assign(m, m + n);
  r.u.assign(u, u + n);
  r.h.assign(h, h + n);
  r.n_steps = n_steps;
  r.dt = dt;
  s->waiting.push_back(r.id);
  *id = r.id;
  s->reqs.emplace(r.id, std::move(r));
  return SPH_OK;
}

sph_status sph_server_set_tick_budget(sph_server* s, int64_t max_particles) {
  if (!s || max_particles < 0) return SPH_E_INVALID;
  s->tick_budget = max_particles;
  return SPH_OK;
}

sph_status sph_server_tick(sph_server* s, int32_t* n_active) {
  if (!s) return SPH_E_INVALID;
  cudaSetDevice(s->device);
  s->st = s->ctx->cur;
  s->eng->st = s->st;
  if (s->intake) s->intake->st = s->st;
  if (n_active) *n_active = 0;
  // admission in submission order while the footprint fits (and the particles
  // stay within the tick budget)
  long long used = 0, parts = 0;
  std::vector<long long> admitted;   // admitted in this tick, with steps to run
  for (long long id : s->resident) {
    used += s->reqs[id].n * kBytesPerParticle;
    parts += s->reqs[id].n;
  }

  while (!s->waiting.empty() && (int)s->resident.size() < s->max_boxes) {
    Request& r = s->reqs[s->waiting.front()];
    if (used + r.n * kBytesPerParticle > s->budget) break;
    if (s->tick_budget > 0 && parts + r.n > s->tick_budget && !s->resident.empty()) break;

    used += r.n * kBytesPerParticle;
    parts += r.n;
    r.state = 1;
    s->resident.push_back(r.id);
    if (r.n_steps > 0) admitted.push_back(r.id);
    s->waiting.pop_front();
  }

  if (s->resident.empty()) return SPH_OK;
  {
    const sph_status is = run_intake(s, admitted);
    if (is != SPH_OK) return is;
  }
  if (s->resident != s->layout) {
    sph_status st = apply_layout(s);
    if (st != SPH_OK) return st;
  }
  sph::Engine& E = *s->eng;
  for (size_t b = 0; b < s->resident.size(); ++b) {
    const Request& r = s->reqs[s->resident[b]];
    E.hbox[b].dt = r.started ? r.dt : 0.0;
  }
  cudaEventRecord(s->e0, s->st);
  sph_status st = E.step_boxes();
  cudaEventRecord(s->e1, s->st);
  if (st != SPH_OK && st != SPH_E_NOT_CONVERGED) return srv_fail(s, st, E.err);
  cudaEventSynchronize(s->e1);
  float ms = 0.0f;
  cudaEventElapsedTime(&ms, s->e0, s->e1);
  if (n_active) *n_active = (int)s->resident.size();
  bool any_done = false;
  for (size_t b = 0; b < s->resident.size(); ++b) {
    Request& r = s->reqs[s->resident[b]];
    if (r.started) {
      r.done_steps++;
      r.step_ms.push_back(ms);
    } else {
      r.started = true;
    }
    if (r.done_steps >= r.n_steps) any_done = true;
  }
  if (any_done) {
    // return the finished boxes; the others stay on the device and move to the
    // new layout at the next tick
    std::vector<long long> keep;
    std::vector<size_t> done;
    for (size_t b = 0; b < s->resident.size(); ++b) {
      Request& r = s->reqs[s->resident[b]];
      if (r.done_steps >= r.n_steps) done.push_back(b);
      else keep.push_back(r.id);
    }
    sph_status fs = finish_many(s, done);
    if (fs != SPH_OK) return fs;
    s->resident = keep;
  }
  return SPH_OK;
}

sph_status sph_server_poll(sph_server* s, int64_t id, int32_t* done, float* step_ms, int32_t max_steps) {
  if (!s || !done) return SPH_E_INVALID;
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return srv_fail(s, SPH_E_INVALID, "unknown request");
  const Request& r = it->second;
  *done = r.state == 2 ? 1 : 0;
  if (step_ms)
    for (int k = 0; k < max_steps && k < (int)r.step_ms.size(); ++k) step_ms[k] = r.step_ms[k];
  return SPH_OK;
}

sph_status sph_server_intake_ms(sph_server* s, int64_t id, float* ms) {
  if (!s || !ms) return SPH_E_INVALID;
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return srv_fail(s, SPH_E_INVALID, "unknown request");
  *ms = it->second.intake_ms;
  return SPH_OK;
}

sph_status sph_server_get(sph_server* s, int64_t id, int field, void* dst, int64_t n) {
  if (!s || !dst) return SPH_E_INVALID;
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return srv_fail(s, SPH_E_INVALID, "unknown request");
  const Request& r = it->second;
  if (r.state != 2) return srv_fail(s, SPH_E_BUSY, "request not finished");
  if (field < 0 || field >= kFields) return srv_fail(s, SPH_E_INVALID, "unknown field");
  const long long want = field == SPH_FIELD_REDUCTIONS ? 8 : r.n;
  if (n != want) return srv_fail(s, SPH_E_INVALID, "n does not match");
  if (r.result[field].empty()) return srv_fail(s, SPH_E_NOT_BUILT, "field not available");
  std::memcpy(dst, r.result[field].data(), r.result[field].size());
  return SPH_OK;
}

sph_status sph_server_release(sph_server* s, int64_t id) {
  if (!s) return SPH_E_INVALID;
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return SPH_E_INVALID;
  if (it->second.state == 1) return srv_fail(s, SPH_E_BUSY, "request is resident");
  if (it->second.state == 0)
    for (auto w = s->waiting.begin(); w != s->waiting.end(); ++w)
      if (*w == id) {
        s->waiting.erase(w);
        break;
      }
  s->reqs.erase(it);
  return SPH_OK;
}

sph_status sph_server_destroy(sph_server* s) {
  if (!s) return SPH_E_INVALID;
  cudaSetDevice(s->device);
  cudaStreamSynchronize(s->st);
  delete s->eng;
  delete s->intake;
  cudaEventDestroy(s->e0);
  cudaEventDestroy(s->e1);
  cudaEventDestroy(s->i0);
  cudaEventDestroy(s->i1);
  if (s->pin) cudaFreeHost(s->pin);
  {
    std::lock_guard<std::mutex> g(s->ctx->mu);
    s->ctx->live--;
  }
  delete s;
  return SPH_OK;
}

}  // extern "C"
