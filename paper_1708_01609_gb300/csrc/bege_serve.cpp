// Serving form of libbege: a request loop with continuous batching.
//
// A server owns one thread and a few CUDA streams.  Requests (strain
// segments from any channel) are queued by bege_serve_submit; the thread
// admits them in arrival order while the device bytes held by admitted
// requests fit the budget, loads each admitted segment's spectrum, cuts its
// correlation with the resident bank into slices of rows, and keeps up to
// `streams` slices in flight, taking slices round-robin over all admitted
// requests.  A request that arrives while others run therefore starts after
// at most one slice and shares the device with them.  Finished requests are
// copied to host memory and their device memory is released at once.
//
// The server drives the device only through the public C ABI of the library
// (bege_load_segment, bege_correlate, bege_query, bege_fetch_tails, ...), so
// every template is computed by exactly the kernels and launch shapes of a
// plain bege_correlate call: results do not depend on what else is served.
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "bege_internal.h"

namespace {

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct Slice {
  int64_t k0 = 0, k1 = 0;
  int32_t job = -1;
  bool done = false;
};

struct Request {
  int64_t id = 0;
  int32_t channel = 0;
  int64_t n = 0;
  std::vector<float> strain;
  int32_t seg = -1;
  std::vector<Slice> slices;
  size_t next = 0;          // next slice to dispatch
  size_t completed = 0;     // slices finished on the device
  int32_t state = 0;        // 0 queued, 1 admitted, 2 done, 3 failed
  int error = 0;
  std::string message;
  double t_submit = 0, t_admit = 0, t_done = 0, gpu_ms = 0;
  uint64_t bytes = 0;       // device bytes charged while admitted
  std::vector<bege_tail> tails;
  int64_t n_tails = 0;
  std::vector<float> sigma;
};

struct Server {
  bege_ctx* ctx = nullptr;
  bege_serve_config cfg{};
  int64_t bank_count = 0, bank_len = 0;
  int device = 0;
  std::vector<cudaStream_t> streams;
  cudaStream_t load_stream = nullptr;
  size_t next_stream = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<int64_t> queue;
  std::map<int64_t, std::unique_ptr<Request>> reqs;
  std::vector<Request*> active;  // admitted and not finished, in admission order
  size_t rr = 0;                 // round-robin position in `active`
  uint64_t held = 0;             // device bytes charged to admitted requests
  int in_flight = 0;
  int64_t next_id = 1;
  bool stop = false;
  std::thread th;
};

// Registry of live servers.  Never destroyed: a server still running when
// the process exits is abandoned with it rather than joined from a static
// destructor.
std::mutex g_reg_mu;
auto* g_servers = new std::map<std::pair<bege_ctx*, int32_t>, std::unique_ptr<Server>>();
int32_t g_next_server = 1;

Server* find_server(bege_ctx* ctx, int32_t id) {
  std::lock_guard<std::mutex> lk(g_reg_mu);
  auto it = g_servers->find({ctx, id});
  return it == g_servers->end() ? nullptr : it->second.get();
}

// Device bytes a segment of length n holds while its request is admitted:
// the spectrum (n/2 + 1 complex) and product coefficients (n/2 float4), plus
// the strain staged during the load.
uint64_t segment_bytes(int64_t n) {
  return (uint64_t)(n / 2 + 1) * 8 + (uint64_t)(n / 2) * 16 + (uint64_t)n * 4;
}

void fail_request(Server* sv, Request* r, int code, const std::string& msg) {
  r->state = 3;
  r->error = code;
  r->message = msg;
  r->t_done = now_s();
  sv->cv_done.notify_all();
}

// Copy one finished slice's tails and sigma to the request's host buffers and
// release its job (its device buffers return to the context's pool at once,
// so a request holds device memory only for its segment and the slices in
// flight).  Called without the server lock: only the server thread touches an
// admitted request's results and device handles until the request is done.
int collect_slice(Server* sv, Request* r, Slice& s) {
  if (r->sigma.empty()) r->sigma.assign((size_t)sv->bank_count, 0.f);
  int64_t nw = 0, nt = 0;
  int rc = bege_fetch_tails(sv->ctx, s.job, nullptr, 0, &nw, &nt);
  if (rc == BEGE_OK || rc == BEGE_EOVERFLOW) {
    const size_t base = r->tails.size();
    r->tails.resize(base + (size_t)nt);
    rc = BEGE_OK;
    if (nt > 0) {
      rc = bege_fetch_tails(sv->ctx, s.job, r->tails.data() + base, nt, &nw, &nt);
      if (rc == BEGE_EOVERFLOW) rc = BEGE_OK;  // the slice kept its first records
      r->tails.resize(base + (size_t)nw);
    }
    r->n_tails += nt;
  }
  if (!rc) rc = bege_get_sigma(sv->ctx, s.job, r->sigma.data() + s.k0, s.k1 - s.k0);
  float ms = 0.f;
  if (bege_job_kernel_ms(sv->ctx, s.job, &ms) == BEGE_OK) r->gpu_ms += ms;
  bege_release(sv->ctx, s.job);
  s.job = -1;
  return rc;
}

void server_loop(Server* sv) {
  cudaSetDevice(sv->device);
  std::unique_lock<std::mutex> lk(sv->mu);
  for (;;) {
    if (sv->stop) {
      // no new slices once stopping; admitted requests finish as failed
      for (Request* r : sv->active)
        if (r->next < r->slices.size()) {
          r->next = r->slices.size();
          if (!r->error) {
            r->error = BEGE_EINVAL;
            r->message = "server stopped";
          }
        }
      if (sv->in_flight == 0 && sv->active.empty()) break;
    }
    bool progress = false;

    // 1. admission, in arrival order, within the budget
    while (!sv->stop && !sv->queue.empty()) {
      Request* r = sv->reqs[sv->queue.front()].get();
      const uint64_t need = segment_bytes(r->n);
      const uint64_t budget = sv->cfg.hbm_budget_bytes;
      if (budget && need > budget) {
        sv->queue.pop_front();
        fail_request(sv, r, BEGE_EBUDGET, "request larger than the server's HBM budget");
        continue;
      }
      if (budget && sv->held + need > budget) break;  // wait for memory to free up
      sv->queue.pop_front();
      lk.unlock();
      int32_t seg = -1;
      const int rc = bege_load_segment(sv->ctx, r->strain.data(), r->n, r->channel,
                                       sv->load_stream, &seg);
      lk.lock();
      if (rc == BEGE_EBUDGET || rc == BEGE_ENOMEM) {
        if (sv->active.empty()) {
          fail_request(sv, r, rc, "no device memory for the request");
          continue;
        }
        sv->queue.push_front(r->id);  // retry once admitted requests finish
        break;
      }
      if (rc) {
        fail_request(sv, r, rc, bege_last_error(sv->ctx));
        continue;
      }
      r->seg = seg;
      r->state = 1;
      r->t_admit = now_s();
      r->bytes = need;
      sv->held += need;
      std::vector<float>().swap(r->strain);
      for (int64_t k = 0; k < sv->bank_count; k += sv->cfg.slice_templates) {
        Slice s;
        s.k0 = k;
        s.k1 = std::min(k + sv->cfg.slice_templates, sv->bank_count);
        r->slices.push_back(s);
      }
      sv->active.push_back(r);
      progress = true;
    }

    // 2. dispatch: slices round-robin over admitted requests
    while (sv->in_flight < sv->cfg.streams) {
      Request* pick = nullptr;
      for (size_t t = 0; t < sv->active.size(); ++t) {
        Request* c = sv->active[(sv->rr + t) % sv->active.size()];
        if (c->next < c->slices.size()) {
          pick = c;
          sv->rr = (sv->rr + t + 1) % sv->active.size();
          break;
        }
      }
      if (!pick) break;
      Slice& s = pick->slices[pick->next];
      cudaStream_t st = sv->streams[sv->next_stream];
      sv->next_stream = (sv->next_stream + 1) % sv->streams.size();
      lk.unlock();
      int32_t job = -1;
      const int rc = bege_correlate(sv->ctx, pick->seg, sv->cfg.bank_id, s.k0, s.k1,
                                    sv->cfg.kappa, st, &job);
      lk.lock();
      if (rc == BEGE_EBUDGET || rc == BEGE_ENOMEM) break;  // retry after something completes
      if (rc) {
        // a failed slice fails its request; slices already in flight still finish
        pick->next = pick->slices.size();
        pick->error = rc;
        pick->message = bege_last_error(sv->ctx);
        break;
      }
      s.job = job;
      ++pick->next;
      ++sv->in_flight;
      progress = true;
    }

    // 3. completions: each finished slice goes to the host right away
    for (size_t ai = 0; ai < sv->active.size(); ++ai) {
      Request* r = sv->active[ai];
      for (size_t i = 0; i < r->next; ++i) {
        Slice& s = r->slices[i];
        if (s.done || s.job < 0) continue;
        if (bege_query(sv->ctx, s.job) == BEGE_ENOTREADY) continue;
        s.done = true;
        --sv->in_flight;
        progress = true;
        lk.unlock();
        const int rc = collect_slice(sv, r, s);
        lk.lock();
        ++r->completed;
        if (rc && !r->error) {
          r->error = rc;
          r->message = bege_last_error(sv->ctx);
        }
      }
    }

    // 4. finished requests: segment released, results handed over
    for (size_t i = 0; i < sv->active.size();) {
      Request* r = sv->active[i];
      size_t live = 0;
      for (size_t j = 0; j < r->next; ++j) live += (r->slices[j].job >= 0);
      if (!(r->next == r->slices.size() && live == 0)) {
        ++i;
        continue;
      }
      sv->active.erase(sv->active.begin() + i);
      if (sv->rr > i) --sv->rr;
      if (!sv->active.empty()) sv->rr %= sv->active.size(); else sv->rr = 0;
      lk.unlock();
      bege_release(sv->ctx, r->seg);
      r->seg = -1;
      lk.lock();
      sv->held -= r->bytes;
      if (r->error) {
        fail_request(sv, r, r->error, r->message.empty() ? "request failed" : r->message);
      } else {
        r->state = 2;
        r->t_done = now_s();
        sv->cv_done.notify_all();
      }
      progress = true;
    }

    if (!progress) sv->cv_work.wait_for(lk, std::chrono::microseconds(200));
  }
}

}  // namespace

extern "C" {

int bege_serve_create(bege_ctx* ctx, const bege_serve_config* cfg, int32_t* server_id) {
  if (!ctx || !cfg || !server_id) return bege::set_last_error(BEGE_EINVAL, "NULL argument");
  if (!std::isfinite(cfg->kappa) || cfg->kappa < 0.f || cfg->reserved != 0.f ||
      cfg->streams < 0 || cfg->slice_templates < 0)
    return bege::set_last_error(BEGE_EINVAL, "bad server configuration");
  const int64_t len = bege_bank_length(ctx, cfg->bank_id);
  const int64_t count = bege::bank_count(ctx, cfg->bank_id);
  if (len <= 0 || count <= 0) return bege::set_last_error(BEGE_EINVAL, "unknown bank handle");
  auto sv = std::make_unique<Server>();
  sv->ctx = ctx;
  sv->cfg = *cfg;
  if (sv->cfg.streams == 0) sv->cfg.streams = 3;
  if (sv->cfg.slice_templates == 0) sv->cfg.slice_templates = 65536;
  sv->bank_count = count;
  sv->bank_len = len;
  sv->device = bege::ctx_device(ctx);
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(sv->device);
  cudaError_t e = cudaStreamCreateWithFlags(&sv->load_stream, cudaStreamNonBlocking);
  for (int i = 0; i < sv->cfg.streams && e == cudaSuccess; ++i) {
    cudaStream_t st = nullptr;
    e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) sv->streams.push_back(st);
  }
  cudaSetDevice(prev);
  if (e != cudaSuccess) {
    for (cudaStream_t st : sv->streams) cudaStreamDestroy(st);
    if (sv->load_stream) cudaStreamDestroy(sv->load_stream);
    return bege::set_last_error(BEGE_ECUDA, cudaGetErrorString(e));
  }
  Server* raw = sv.get();
  int32_t id;
  {
    std::lock_guard<std::mutex> lk(g_reg_mu);
    id = g_next_server++;
    (*g_servers)[{ctx, id}] = std::move(sv);
  }
  raw->th = std::thread(server_loop, raw);
  *server_id = id;
  return BEGE_OK;
}

int bege_serve_submit(bege_ctx* ctx, int32_t server_id, const float* strain, int64_t n,
                      int32_t channel, int64_t* request_id) {
  Server* sv = find_server(ctx, server_id);
  if (!sv || !strain || !request_id) return bege::set_last_error(BEGE_EINVAL, "bad argument");
  if (n < 1024 || n > (1 << 17) || (n & (n - 1)) || n < sv->bank_len)
    return bege::set_last_error(BEGE_EINVAL,
                                "n must be a power of two in [2^10, 2^17], >= template length");
  auto r = std::make_unique<Request>();
  r->channel = channel;
  r->n = n;
  r->strain.assign(strain, strain + n);
  r->t_submit = now_s();
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->stop) return bege::set_last_error(BEGE_EINVAL, "server is stopping");
    r->id = sv->next_id++;
    *request_id = r->id;
    sv->queue.push_back(r->id);
    sv->reqs[r->id] = std::move(r);
  }
  sv->cv_work.notify_one();
  return BEGE_OK;
}

int bege_serve_wait(bege_ctx* ctx, int32_t server_id, int64_t request_id, int32_t timeout_ms) {
  Server* sv = find_server(ctx, server_id);
  if (!sv) return bege::set_last_error(BEGE_EINVAL, "unknown server");
  std::unique_lock<std::mutex> lk(sv->mu);
  auto it = sv->reqs.find(request_id);
  if (it == sv->reqs.end()) return bege::set_last_error(BEGE_EINVAL, "unknown request");
  Request* r = it->second.get();
  auto finished = [&] { return r->state >= 2; };
  if (timeout_ms < 0) {
    sv->cv_done.wait(lk, finished);
  } else if (!sv->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), finished)) {
    return bege::set_last_error(BEGE_ETIMEDOUT, "request not finished");
  }
  if (r->state == 3) return bege::set_last_error(r->error, r->message);
  return BEGE_OK;
}

int bege_serve_info_get(bege_ctx* ctx, int32_t server_id, int64_t request_id,
                        bege_serve_info* info) {
  Server* sv = find_server(ctx, server_id);
  if (!sv || !info) return bege::set_last_error(BEGE_EINVAL, "bad argument");
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->reqs.find(request_id);
  if (it == sv->reqs.end()) return bege::set_last_error(BEGE_EINVAL, "unknown request");
  const Request* r = it->second.get();
  info->state = r->state;
  info->channel = r->channel;
  info->n = r->n;
  info->n_tails = r->n_tails;
  info->t_submit = r->t_submit;
  info->t_admit = r->t_admit;
  info->t_done = r->t_done;
  info->gpu_ms = r->gpu_ms;
  return BEGE_OK;
}

int bege_serve_fetch_tails(bege_ctx* ctx, int32_t server_id, int64_t request_id, bege_tail* out,
                           int64_t capacity, int64_t* n_written, int64_t* n_total) {
  Server* sv = find_server(ctx, server_id);
  if (!sv || !n_written || !n_total || capacity < 0 || (capacity > 0 && !out))
    return bege::set_last_error(BEGE_EINVAL, "bad argument");
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->reqs.find(request_id);
  if (it == sv->reqs.end()) return bege::set_last_error(BEGE_EINVAL, "unknown request");
  const Request* r = it->second.get();
  if (r->state != 2) return bege::set_last_error(BEGE_ENOTREADY, "request not done");
  const int64_t have = (int64_t)r->tails.size();
  const int64_t nc = std::min(have, capacity);
  if (nc) std::copy(r->tails.begin(), r->tails.begin() + nc, out);
  *n_written = nc;
  *n_total = r->n_tails;
  if (nc < r->n_tails) return bege::set_last_error(BEGE_EOVERFLOW, "more tails than copied");
  return BEGE_OK;
}

int bege_serve_get_sigma(bege_ctx* ctx, int32_t server_id, int64_t request_id, float* out,
                         int64_t count) {
  Server* sv = find_server(ctx, server_id);
  if (!sv || !out) return bege::set_last_error(BEGE_EINVAL, "bad argument");
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->reqs.find(request_id);
  if (it == sv->reqs.end()) return bege::set_last_error(BEGE_EINVAL, "unknown request");
  const Request* r = it->second.get();
  if (r->state != 2) return bege::set_last_error(BEGE_ENOTREADY, "request not done");
  if (count != (int64_t)r->sigma.size())
    return bege::set_last_error(BEGE_EINVAL, "count must equal the bank size");
  std::copy(r->sigma.begin(), r->sigma.end(), out);
  return BEGE_OK;
}

int bege_serve_forget(bege_ctx* ctx, int32_t server_id, int64_t request_id) {
  Server* sv = find_server(ctx, server_id);
  if (!sv) return bege::set_last_error(BEGE_EINVAL, "unknown server");
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->reqs.find(request_id);
  if (it == sv->reqs.end()) return bege::set_last_error(BEGE_EINVAL, "unknown request");
  if (it->second->state < 2) return bege::set_last_error(BEGE_ENOTREADY, "request not done");
  sv->reqs.erase(it);
  return BEGE_OK;
}

int bege_serve_destroy(bege_ctx* ctx, int32_t server_id) {
  std::unique_ptr<Server> sv;
  {
    std::lock_guard<std::mutex> lk(g_reg_mu);
    auto it = g_servers->find({ctx, server_id});
    if (it == g_servers->end()) return bege::set_last_error(BEGE_EINVAL, "unknown server");
    sv = std::move(it->second);
    g_servers->erase(it);
  }
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
    // queued requests that were never admitted are dropped
    for (int64_t id : sv->queue) {
      Request* r = sv->reqs[id].get();
      r->state = 3;
      r->error = BEGE_EINVAL;
      r->message = "server stopped";
    }
    sv->queue.clear();
  }
  sv->cv_work.notify_all();
  sv->cv_done.notify_all();
  if (sv->th.joinable()) sv->th.join();
  // requests still admitted after the last slice (none: the loop drains them)
  for (cudaStream_t st : sv->streams) cudaStreamDestroy(st);
  if (sv->load_stream) cudaStreamDestroy(sv->load_stream);
  return BEGE_OK;
}

}  // extern "C"

namespace bege {
// Stop every server of a context (called by bege_destroy before it frees the
// context's device memory).
void serve_destroy_all(bege_ctx* ctx) {
  std::vector<int32_t> ids;
  {
    std::lock_guard<std::mutex> lk(g_reg_mu);
    for (auto& kv : *g_servers)
      if (kv.first.first == ctx) ids.push_back(kv.first.second);
  }
  for (int32_t id : ids) bege_serve_destroy(ctx, id);
}
}  // namespace bege
