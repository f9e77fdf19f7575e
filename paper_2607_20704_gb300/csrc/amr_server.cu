// amr_server.cu -- continuous-batching serving loop over the level-advance
// library (include/amr.h, amr_server_*).
//
// Requests (one mesh, a number of coarse steps, a precision) are queued by
// amr_server_submit.  A scheduler thread admits, in arrival order, every
// queued request that fits the device budget (a request that does not fit
// waits without holding back later ones): it joins a running wave of its
// precision that has a free member slot, else it starts a new wave while
// wave slots remain.  A wave is one batched handle on a stream of its own,
// in which every member stops after its own number of coarse steps (the
// handle's per-member step counters); waves overlap on the GPU.  Each wave
// keeps at most two coarse steps in flight; a CUDA event per coarse step
// tells the scheduler when members are finished, and their final state is
// copied to host memory.  Between coarse steps a wave is repacked
// (amr_batch_repack) when requests wait to join it or when finished members
// hold a quarter of its octs: finished members are dropped, their device
// memory and budget return, joining requests are added, and the members that
// keep running continue bit for bit as they would alone.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "amr.h"

void amr_set_error_text(const char *text);

namespace {

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

amr_status set_error(amr_status s, const std::string &msg) {
  amr_set_error_text(msg.c_str());
  return s;
}

struct Request {
  int64_t id = 0;
  int levelmin = 1, levelmax = 1, steps = 1, precision = 8;
  double gamma = 1.4, cfl = 0.8, smallr = 1e-10, smallc = 1e-10;
  std::vector<uint8_t> level;
  std::vector<uint32_t> i, j, k;
  std::vector<uint64_t> hk;
  std::vector<double> U;
  size_t est_bytes = 0;
  double t_submit = 0, t_admit = -1, t_done = -1;
  double work = 0;  // leaf cell-updates of the whole solve
  bool done = false, failed = false;
  bool solo = false;  // admitted alone (its wave-mates' batch could not be built)
  std::string error;
  std::vector<std::vector<uint64_t>> keys;  // final state, per level
  std::vector<std::vector<double>> Uout;
};

struct Wave {
  amr_handle h = nullptr;
  cudaStream_t s = nullptr;
  int precision = 8;
  std::vector<Request *> reqs;     // members, in the handle's member order
  std::vector<int> joined;         // coarse steps the wave had completed when each joined
  std::vector<Request *> joiners;  // admitted, to be added at the next repack
  int issued = 0, completed = 0;
  std::vector<cudaEvent_t> ev;
  size_t bytes = 0;        // device bytes of the handle
  size_t reserved = 0;     // budget held for the joiners
  bool want_repack = false;
};

// device bytes of a handle per oct, for admission before the handle exists
// (state with ghosts, level-step scratch, index, hash, create-time staging)
struct Request;
size_t need_bytes(const std::vector<Request *> &rs);

size_t estimate_bytes(int64_t n_oct, int precision) {
  const size_t w = precision == 4 ? 4 : 8;
  return size_t(n_oct) * (w * (8 * 5 * 2 + 8 * 40) + 1024) + (8u << 20);
}

size_t need_bytes(const std::vector<Request *> &rs) {
  size_t b = 0;
  for (auto *r : rs) b += r->est_bytes;
  return b;
}

}  // namespace

struct amr_server {
  amr_server_params p{};
  int device = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request *> queue;
  std::unordered_map<int64_t, std::unique_ptr<Request>> reqs;
  std::vector<Wave *> waves;  // scheduler thread only
  std::thread th;
  std::atomic<bool> stop{false};
  int64_t next_id = 1;
  size_t bytes_in_use = 0;
  int64_t submitted = 0, admitted = 0, completed = 0, failed = 0;
  double cell_updates = 0, first_submit = -1, last_done = -1;
  std::vector<double> latencies, queue_waits;
  std::string fatal;

  void loop();
  bool admit();
  void start_wave(std::vector<Request *> take);
  bool progress(Wave *w);
  void repack(Wave *w);
  void finish_member(Wave *w, Request *r, int member);
  void joined_now(Wave *w, Request *r, int member, double t);
};

namespace {

amr_member member_of(const Request *r) {
  amr_member m{};
  m.levelmin = r->levelmin;
  m.levelmax = r->levelmax;
  m.gamma = r->gamma;
  m.cfl = r->cfl;
  m.smallr = r->smallr;
  m.smallc = r->smallc;
  m.n_oct = int64_t(r->level.size());
  m.level = r->level.data();
  m.i = r->i.data();
  m.j = r->j.data();
  m.k = r->k.data();
  m.hilbert_key = r->hk.empty() ? nullptr : r->hk.data();
  m.U = r->U.data();
  return m;
}

}  // namespace

// bookkeeping of a request that has just become member `member` of a wave
// (mu held)
void amr_server::joined_now(Wave *w, Request *r, int member, double t) {
  r->t_admit = t;
  ++admitted;
  queue_waits.push_back(1e3 * (t - r->t_submit));
  amr_select_member(w->h, member);
  amr_info mi;
  amr_get_info(w->h, &mi);
  double per_step = 0;
  for (int l = r->levelmin; l <= 15; ++l)
    if (mi.level_octs[l]) per_step += double(mi.level_leaf_cells[l]) * double(int64_t(1) << (l - r->levelmin));
  r->work = per_step * r->steps;
}

// Admission, in arrival order: every queued request whose estimated bytes
// fit the remaining budget joins a running wave of its precision with a
// free member slot, or starts a new wave (with the other new requests of
// its precision) while wave slots remain.  A request marked solo starts a
// wave of its own.
bool amr_server::admit() {
  std::vector<std::vector<Request *>> groups;
  {
    std::lock_guard<std::mutex> g(mu);
    if (queue.empty()) return false;
    size_t left = p.hbm_budget_bytes > bytes_in_use ? p.hbm_budget_bytes - bytes_in_use : 0;
    int slots = p.max_waves - int(waves.size());
    int open[2] = {-1, -1};  // the new group of each precision
    for (auto it = queue.begin(); it != queue.end();) {
      Request *r = *it;
      if (r->est_bytes > left) {
        ++it;
        continue;
      }
      Wave *w = nullptr;
      if (!r->solo)
        for (Wave *x : waves)
          if (x->precision == r->precision && int(x->reqs.size() + x->joiners.size()) < p.max_wave_members) {
            w = x;
            break;
          }
      const int pi = r->precision == 8 ? 1 : 0;
      if (w) {
        w->joiners.push_back(r);
        w->reserved += r->est_bytes;
      } else if (!r->solo && open[pi] >= 0 && int(groups[size_t(open[pi])].size()) < p.max_wave_members) {
        groups[size_t(open[pi])].push_back(r);
      } else if (slots > 0) {
        --slots;
        groups.push_back({r});
        if (!r->solo) open[pi] = int(groups.size()) - 1;
      } else {
        ++it;
        continue;
      }
      left -= r->est_bytes;
      bytes_in_use += r->est_bytes;
      it = queue.erase(it);
    }
  }
  for (auto &gq : groups) start_wave(gq);
  return !groups.empty();
}

void amr_server::start_wave(std::vector<Request *> take) {
  Wave *w = new Wave();
  w->reqs = take;
  w->precision = take[0]->precision;
  size_t est = 0;
  for (auto *r : take) est += r->est_bytes;
  cudaStreamCreateWithFlags(&w->s, cudaStreamNonBlocking);
  amr_params prm;
  amr_params_default(&prm);
  prm.precision = w->precision;
  prm.stream = w->s;
  prm.tile = p.tile ? p.tile : 128;
  prm.schedule = p.schedule >= 0 ? p.schedule : 0;
  std::vector<amr_member> mem(take.size());
  std::vector<int32_t> steps(take.size());
  for (size_t q = 0; q < take.size(); ++q) {
    mem[q] = member_of(take[q]);
    steps[q] = take[q]->steps;
  }
  amr_status s = amr_create_batch(&prm, int(take.size()), mem.data(), &w->h);
  if (s == AMR_OK) s = amr_set_member_steps(w->h, steps.data(), int(steps.size()));
  const double t = now_s();
  std::lock_guard<std::mutex> g(mu);
  if (s != AMR_OK && take.size() > 1) {
    // one of the meshes is invalid (or the batch too large): retry each
    // request alone, in the same order, so that only the bad one fails
    if (w->h) amr_destroy(w->h);
    cudaStreamDestroy(w->s);
    delete w;
    bytes_in_use -= std::min(bytes_in_use, est);
    for (auto it = take.rbegin(); it != take.rend(); ++it) {
      (*it)->solo = true;
      queue.push_front(*it);
    }
    return;
  }
  if (s != AMR_OK) {
    // the request fails with the handle's error; its budget returns
    const std::string msg = amr_last_error();
    for (auto *r : take) {
      r->failed = r->done = true;
      r->error = msg;
      r->t_done = t;
      ++failed;
    }
    bytes_in_use -= std::min(bytes_in_use, est);
    if (w->h) amr_destroy(w->h);
    cudaStreamDestroy(w->s);
    delete w;
    cv_done.notify_all();
    return;
  }
  amr_info inf;
  amr_get_info(w->h, &inf);
  // account the handle's real footprint instead of the estimate
  bytes_in_use = bytes_in_use - std::min(bytes_in_use, est) + size_t(inf.device_bytes);
  w->bytes = size_t(inf.device_bytes);
  w->joined.assign(take.size(), 0);
  for (size_t q = 0; q < take.size(); ++q) joined_now(w, take[q], int(q), t);
  waves.push_back(w);
}

void amr_server::finish_member(Wave *w, Request *r, int member) {
  // a non-finite state fails its own request only
  std::vector<int32_t> errs(w->reqs.size());
  amr_status s = amr_member_errors(w->h, errs.data(), int(errs.size()));
  if (s == AMR_OK && errs[member]) {
    std::lock_guard<std::mutex> g(mu);
    r->failed = r->done = true;
    r->error = "non-finite state";
    r->t_done = now_s();
    ++failed;
    cv_done.notify_all();
    return;
  }
  amr_select_member(w->h, member);
  std::vector<std::vector<uint64_t>> keys(16);
  std::vector<std::vector<double>> U(16);
  for (int l = 0; l <= 15 && s == AMR_OK; ++l) {
    int64_t n = 0;
    s = amr_read(w->h, l, &n, nullptr, nullptr, 0);
    if (s != AMR_OK || n == 0) continue;
    keys[l].resize(n);
    U[l].resize(40 * size_t(n));
    s = amr_read(w->h, l, &n, keys[l].data(), U[l].data(), n);
  }
  const double t = now_s();
  std::lock_guard<std::mutex> g(mu);
  r->keys = std::move(keys);
  r->Uout = std::move(U);
  r->t_done = t;
  r->done = true;
  if (s != AMR_OK) {
    r->failed = true;
    r->error = amr_last_error();
    ++failed;
  } else {
    ++completed;
    latencies.push_back(1e3 * (t - r->t_submit));
    cell_updates += r->work;
    last_done = t;
  }
  cv_done.notify_all();
}

// Between coarse steps: drop the finished members, add the joiners.  If the
// joiners cannot be added together (an invalid mesh among them), they are
// added one at a time and only the invalid one fails.
void amr_server::repack(Wave *w) {
  std::vector<int32_t> keep;
  std::vector<Request *> reqs;
  std::vector<int> joined;
  for (size_t q = 0; q < w->reqs.size(); ++q)
    if (!w->reqs[q]->done) {
      keep.push_back(int32_t(q));
      reqs.push_back(w->reqs[q]);
      joined.push_back(w->joined[q]);
    }
  std::vector<Request *> add = w->joiners;
  std::vector<amr_member> mem;
  std::vector<int32_t> steps;
  for (auto *r : add) {
    mem.push_back(member_of(r));
    steps.push_back(r->steps);
  }
  std::vector<Request *> joined_ok, joined_bad;
  std::string bad_msg;
  amr_status s = keep.empty() && add.empty()
                     ? AMR_OK
                     : amr_batch_repack(w->h, int(keep.size()), keep.data(), int(add.size()), mem.data(),
                                        steps.data());
  if (s == AMR_OK) {
    joined_ok = add;
  } else {
    // drop the finished members first, then try the joiners one by one
    s = keep.empty() ? AMR_OK : amr_batch_repack(w->h, int(keep.size()), keep.data(), 0, nullptr, nullptr);
    if (s != AMR_OK) {
      // the wave itself cannot be rebuilt: its running members fail
      const std::string msg = amr_last_error();
      std::lock_guard<std::mutex> g(mu);
      for (auto *r : reqs) {
        r->failed = r->done = true;
        r->error = msg;
        r->t_done = now_s();
        ++failed;
      }
      for (auto *r : add) {
        r->failed = r->done = true;
        r->error = msg;
        r->t_done = now_s();
        ++failed;
      }
      reqs.clear();
      joined.clear();
      add.clear();
      w->joiners.clear();
      cv_done.notify_all();
    } else {
      for (size_t q = 0; q < add.size(); ++q) {
        std::vector<int32_t> all;
        for (size_t t = 0; t < reqs.size() + joined_ok.size(); ++t) all.push_back(int32_t(t));
        amr_status sj = amr_batch_repack(w->h, int(all.size()), all.data(), 1, &mem[q], &steps[q]);
        if (sj == AMR_OK) {
          joined_ok.push_back(add[q]);
        } else {
          joined_bad.push_back(add[q]);
          bad_msg = amr_last_error();
        }
      }
    }
  }
  const double t = now_s();
  amr_info inf;
  amr_get_info(w->h, &inf);
  std::lock_guard<std::mutex> g(mu);
  for (auto *r : joined_bad) {
    r->failed = r->done = true;
    r->error = bad_msg;
    r->t_done = t;
    ++failed;
  }
  bytes_in_use -= std::min(bytes_in_use, w->bytes + w->reserved);
  w->reserved = 0;
  w->joiners.clear();
  w->reqs = reqs;
  w->joined = joined;
  for (auto *r : joined_ok) {
    w->reqs.push_back(r);
    w->joined.push_back(w->completed);
    joined_now(w, r, int(w->reqs.size()) - 1, t);
  }
  w->bytes = w->reqs.empty() ? 0 : size_t(inf.device_bytes);
  bytes_in_use += w->bytes;
  if (!joined_bad.empty()) cv_done.notify_all();
}

// Finish members whose steps are done, repack when joiners wait or finished
// members hold a quarter of the octs (once the wave is idle), issue coarse
// steps (at most two in flight); true when the wave has nothing left.
bool amr_server::progress(Wave *w) {
  while (w->completed < int(w->ev.size()) && cudaEventQuery(w->ev[w->completed]) == cudaSuccess)
    ++w->completed;
  int64_t fin_octs = 0, all_octs = 0;
  bool running = false;
  for (size_t q = 0; q < w->reqs.size(); ++q) {
    Request *r = w->reqs[q];
    if (!r->done && w->completed - w->joined[q] >= r->steps) finish_member(w, r, int(q));
    const int64_t n = int64_t(r->level.size());
    all_octs += n;
    if (r->done)
      fin_octs += n;
    else
      running = true;
  }
  bool want_repack;
  {
    std::lock_guard<std::mutex> g(mu);
    if (!running && w->joiners.empty()) return true;
    want_repack = !w->joiners.empty() || (fin_octs > 0 && 4 * fin_octs >= all_octs);
  }
  if (want_repack) {
    if (w->issued != w->completed) return false;  // let the steps in flight finish
    repack(w);
    if (w->reqs.empty()) return true;
  }
  int need = 0;
  for (size_t q = 0; q < w->reqs.size(); ++q)
    if (!w->reqs[q]->done) need = std::max(need, w->joined[q] + w->reqs[q]->steps - w->issued);
  while (need > 0 && w->issued - w->completed < 2) {
    if (amr_advance(w->h, 1, nullptr) != AMR_OK) {
      const std::string msg = amr_last_error();
      std::lock_guard<std::mutex> g(mu);
      for (auto *r : w->reqs)
        if (!r->done) {
          r->failed = r->done = true;
          r->error = msg;
          ++failed;
        }
      cv_done.notify_all();
      return true;
    }
    cudaEvent_t e;
    cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
    cudaEventRecord(e, w->s);
    w->ev.push_back(e);
    ++w->issued;
    --need;
  }
  return false;
}

void amr_server::loop() {
  cudaSetDevice(device);
  while (true) {
    bool busy = false;
    while (admit()) busy = true;
    for (size_t t = 0; t < waves.size();) {
      Wave *w = waves[t];
      if (progress(w)) {
        cudaStreamSynchronize(w->s);
        amr_destroy(w->h);
        for (auto e : w->ev) cudaEventDestroy(e);
        cudaStreamDestroy(w->s);
        {
          std::lock_guard<std::mutex> g(mu);
          bytes_in_use -= std::min(bytes_in_use, w->bytes + w->reserved);
          // joiners of a wave that ended before their repack go back to the queue
          for (auto it = w->joiners.rbegin(); it != w->joiners.rend(); ++it) queue.push_front(*it);
        }
        delete w;
        waves.erase(waves.begin() + t);
        busy = true;
      } else {
        ++t;
      }
    }
    std::unique_lock<std::mutex> lk(mu);
    if (stop && queue.empty() && waves.empty()) break;
    if (!busy)
      cv_work.wait_for(lk, std::chrono::microseconds(waves.empty() ? 2000 : 100));
  }
}

extern "C" amr_status amr_server_create(const amr_server_params *p, amr_server_t *out) {
  if (!out) return set_error(AMR_EINVAL, "amr_server_create: out is NULL");
  *out = nullptr;
  amr_server *s = new amr_server();
  if (p) s->p = *p;
  if (s->p.hbm_budget_bytes == 0) s->p.hbm_budget_bytes = size_t(120) * 1000 * 1000 * 1000;
  if (s->p.max_waves <= 0) s->p.max_waves = 8;
  if (s->p.max_wave_members <= 0) s->p.max_wave_members = 256;
  if (s->p.device < 0) cudaGetDevice(&s->device); else s->device = s->p.device;
  s->th = std::thread([s] { s->loop(); });
  *out = s;
  return AMR_OK;
}

extern "C" amr_status amr_server_submit(amr_server_t s, const amr_request *req, int64_t *id_out) {
  if (!s || !req || !id_out) return set_error(AMR_EINVAL, "amr_server_submit: NULL argument");
  const amr_member &m = req->mesh;
  if (!m.level || !m.i || !m.j || !m.k || !m.U || m.n_oct < 1)
    return set_error(AMR_EINVAL, "amr_server_submit: empty or NULL mesh");
  if (req->n_coarse_steps < 1) return set_error(AMR_EINVAL, "amr_server_submit: n_coarse_steps < 1");
  if (req->precision != 4 && req->precision != 8)
    return set_error(AMR_EINVAL, "amr_server_submit: precision must be 4 or 8");
  auto r = std::make_unique<Request>();
  r->levelmin = m.levelmin;
  r->levelmax = m.levelmax;
  r->gamma = m.gamma;
  r->cfl = m.cfl;
  r->smallr = m.smallr;
  r->smallc = m.smallc;
  r->steps = req->n_coarse_steps;
  r->precision = req->precision;
  const int64_t n = m.n_oct;
  r->level.assign(m.level, m.level + n);
  r->i.assign(m.i, m.i + n);
  r->j.assign(m.j, m.j + n);
  r->k.assign(m.k, m.k + n);
  if (m.hilbert_key) r->hk.assign(m.hilbert_key, m.hilbert_key + n);
  r->U.assign(m.U, m.U + 40 * n);
  r->est_bytes = estimate_bytes(n, r->precision);
  if (r->est_bytes > s->p.hbm_budget_bytes)
    return set_error(AMR_ENOMEM, "amr_server_submit: the request alone exceeds the device budget");
  std::lock_guard<std::mutex> g(s->mu);
  r->id = s->next_id++;
  r->t_submit = now_s();
  if (s->first_submit < 0) s->first_submit = r->t_submit;
  *id_out = r->id;
  s->queue.push_back(r.get());
  s->reqs[r->id] = std::move(r);
  ++s->submitted;
  s->cv_work.notify_all();
  return AMR_OK;
}

extern "C" amr_status amr_server_wait(amr_server_t s, int64_t id, double timeout_s, int *done) {
  if (!s) return set_error(AMR_EINVAL, "amr_server_wait: NULL server");
  std::unique_lock<std::mutex> lk(s->mu);
  auto ready = [&] {
    if (id < 0) return s->completed + s->failed == s->submitted;
    auto it = s->reqs.find(id);
    return it == s->reqs.end() || it->second->done;
  };
  if (id >= 0 && !s->reqs.count(id)) return set_error(AMR_EINVAL, "amr_server_wait: unknown request");
  bool ok;
  if (timeout_s < 0)
    s->cv_done.wait(lk, ready), ok = true;
  else
    ok = s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), ready);
  if (done) *done = ok ? 1 : 0;
  if (ok && id >= 0 && s->reqs[id]->failed)
    return set_error(AMR_ECUDA, "request " + std::to_string(id) + " failed: " + s->reqs[id]->error);
  return AMR_OK;
}

extern "C" amr_status amr_server_read(amr_server_t s, int64_t id, int level, int64_t *n_oct,
                                      uint64_t *keys, double *U, int64_t cap) {
  if (!s) return set_error(AMR_EINVAL, "amr_server_read: NULL server");
  if (level < 0 || level > 15) return set_error(AMR_EINVAL, "amr_server_read: bad level");
  std::lock_guard<std::mutex> g(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return set_error(AMR_EINVAL, "amr_server_read: unknown request");
  Request *r = it->second.get();
  if (!r->done || r->failed) return set_error(AMR_EINVAL, "amr_server_read: request not finished");
  const int64_t n = int64_t(r->keys[level].size());
  if (n_oct) *n_oct = n;
  if ((keys || U) && cap < n) return set_error(AMR_EINVAL, "amr_server_read: cap too small");
  if (keys && n) std::memcpy(keys, r->keys[level].data(), 8 * n);
  if (U && n) std::memcpy(U, r->Uout[level].data(), sizeof(double) * 40 * n);
  return AMR_OK;
}

extern "C" amr_status amr_server_release(amr_server_t s, int64_t id) {
  if (!s) return set_error(AMR_EINVAL, "amr_server_release: NULL server");
  std::lock_guard<std::mutex> g(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end() || !it->second->done)
    return set_error(AMR_EINVAL, "amr_server_release: unknown or unfinished request");
  s->reqs.erase(it);
  return AMR_OK;
}

static double percentile(std::vector<double> v, double q) {
  if (v.empty()) return 0.0;
  std::sort(v.begin(), v.end());
  const double pos = q * double(v.size() - 1);
  const size_t a = size_t(pos);
  const size_t b = std::min(a + 1, v.size() - 1);
  return v[a] + (v[b] - v[a]) * (pos - double(a));
}

extern "C" amr_status amr_server_get_stats(amr_server_t s, amr_server_stats *st) {
  if (!s || !st) return set_error(AMR_EINVAL, "amr_server_get_stats: NULL argument");
  std::lock_guard<std::mutex> g(s->mu);
  std::memset(st, 0, sizeof *st);
  st->submitted = s->submitted;
  st->admitted = s->admitted;
  st->completed = s->completed;
  st->failed = s->failed;
  st->queued = int64_t(s->queue.size());
  st->running_waves = int64_t(s->waves.size());
  st->latency_p50_ms = percentile(s->latencies, 0.50);
  st->latency_p99_ms = percentile(s->latencies, 0.99);
  double sum = 0;
  for (double x : s->latencies) sum += x;
  st->latency_mean_ms = s->latencies.empty() ? 0.0 : sum / double(s->latencies.size());
  st->queue_p50_ms = percentile(s->queue_waits, 0.50);
  st->cell_updates = s->cell_updates;
  st->span_s = (s->last_done > 0 && s->first_submit > 0) ? s->last_done - s->first_submit : 0.0;
  st->device_bytes = int64_t(s->bytes_in_use);
  return AMR_OK;
}

extern "C" amr_status amr_server_destroy(amr_server_t s) {
  if (!s) return AMR_OK;
  {
    std::lock_guard<std::mutex> g(s->mu);
    s->stop = true;
    s->cv_work.notify_all();
  }
  if (s->th.joinable()) s->th.join();
  delete s;
  return AMR_OK;
}
