// Request loop for catalogue queries arriving over time (a mock-ensemble
// covariance campaign): continuous batching with admission by device
// memory.
//
// Two host threads share the GPU through two streams:
//  * the builder takes pending requests in arrival order, admits one while
//    the graphs held on the device stay within the budget (always when
//    nothing is held, so a request larger than the budget still runs
//    alone), copies its inputs, builds its graph and fixed-point weights on
//    the build stream and hands it to the counter;
//  * the counter takes every ready request: 3pCF requests with the same
//    bin count and weighting go into one batched persistent launch
//    (gs_count_3pcf_batch's kernel), 4pCF requests run one by one; results
//    are copied to the caller's buffers, graphs are freed and waiters woken.
// Building the next requests overlaps counting the current ones on the
// device. Every result equals the single-request result exactly: counts are
// integers and weighted sums are exact before their one rounding.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <thread>

#include "gs_internal.cuh"

namespace gs {
namespace {

double now_s(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

struct Job {
  int64_t ticket = 0;
  gs_request req{};
  std::vector<int32_t> xyz;
  std::vector<int64_t> edges;
  std::vector<float> w;
  int status = GS_OK;
  bool done = false;
  double t_submit = 0, t_start = 0, t_done = 0;
  // built state
  gs_graph* graph = nullptr;
  std::unique_ptr<Scratch> wscratch;  // owns the fixed-point weights
  FixedW fw;
  int64_t bytes = 0;  // device bytes held while admitted
};

}  // namespace
}  // namespace gs

struct gs_server {
  gs_server_config cfg{};
  int device = 0;
  std::chrono::steady_clock::time_point t0;
  std::mutex mu;
  std::condition_variable cv_pending, cv_ready, cv_done, cv_mem;
  std::deque<std::shared_ptr<gs::Job>> pending, ready;
  std::map<int64_t, std::shared_ptr<gs::Job>> jobs;
  int64_t next_ticket = 1;
  int64_t held_bytes = 0;
  int in_flight = 0;
  bool stop = false;
  cudaStream_t s_build = nullptr, s_count = nullptr;
  std::thread builder, counter;
};

namespace gs {
namespace {

int64_t estimate_bytes(const gs_request& r) {
  // points (28 B) plus the oriented edges of a uniform catalogue at the
  // request's mean density, doubled for clustering
  const double n = (double)r.n;
  double edges = 0.0;
  if (r.box_u > 0 && r.n > 1) {
    const double rmax = (double)r.edges_u[r.nb];
    const double vol = (double)r.box_u * (double)r.box_u * (double)r.box_u;
    edges = n * (n - 1) / 2.0 * (4.18879020478639 * rmax * rmax * rmax / vol);
  } else {
    edges = n * 64.0;
  }
  return (int64_t)(28.0 * n + 2.0 * 4.0 * edges) + (1 << 20);
}

void finish(gs_server* S, const std::shared_ptr<Job>& j, int status) {
  if (j->graph) {
    gs_free_graph(j->graph);
    j->graph = nullptr;
  }
  j->wscratch.reset();
  std::lock_guard<std::mutex> lk(S->mu);
  j->status = status;
  j->done = true;
  j->t_done = now_s(S->t0);
  S->held_bytes -= j->bytes;
  j->bytes = 0;
  S->in_flight -= 1;
  S->cv_done.notify_all();
  S->cv_mem.notify_all();
}

void builder_loop(gs_server* S) {
  cudaSetDevice(S->device);
  for (;;) {
    std::shared_ptr<Job> j;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv_pending.wait(lk, [&] { return S->stop || !S->pending.empty(); });
      if (S->stop) return;
      j = S->pending.front();
      const int64_t est = estimate_bytes(j->req);
      // admission: wait until the estimate fits next to the held graphs
      S->cv_mem.wait(lk, [&] {
        return S->stop || S->held_bytes == 0 || S->held_bytes + est <= (int64_t)S->cfg.device_budget_bytes;
      });
      if (S->stop) return;
      S->pending.pop_front();
      S->held_bytes += est;
      j->bytes = est;
      j->t_start = now_s(S->t0);
    }
    gs_options o{};
    o.stream = S->s_build;
    int st = gs_build_graph(j->xyz.data(), j->req.n, j->req.box_u, j->edges.data(), j->req.nb, &o,
                            &j->graph);
    if (!st && !j->w.empty()) {
      j->wscratch.reset(new (std::nothrow) Scratch(S->s_build));
      if (!j->wscratch) st = GS_ENOMEM;
      else st = prepare_weights(j->graph->g, j->w.data(), &j->fw, *j->wscratch, S->s_build);
      if (!st) st = cuda_status(cudaStreamSynchronize(S->s_build));
    }
    if (st) {
      finish(S, j, st);
      continue;
    }
    {
      std::lock_guard<std::mutex> lk(S->mu);
      // replace the estimate by what the graph actually holds
      S->held_bytes += j->graph->g.device_bytes + 8 * j->req.n - j->bytes;
      j->bytes = j->graph->g.device_bytes + 8 * j->req.n;
      S->ready.push_back(j);
      S->cv_ready.notify_all();
    }
  }
}

int run_3pcf_batch(gs_server* S, std::vector<std::shared_ptr<Job>>& batch) {
  const int ng = (int)batch.size();
  const int nb = batch[0]->req.nb;
  const int64_t nc = num_conf3(nb);
  const bool weighted = !batch[0]->w.empty();
  Opts o;
  o.stream = S->s_count;
  Scratch sc(o.stream);
  std::vector<const Graph*> gr(ng);
  std::vector<FixedW> fws(weighted ? ng : 0);
  std::vector<uint64_t*> dc(ng);
  std::vector<double*> dw(ng, nullptr);
  for (int k = 0; k < ng; ++k) {
    gr[k] = &batch[k]->graph->g;
    if (weighted) fws[k] = batch[k]->fw;
    dc[k] = sc.alloc<uint64_t>(nc);
    if (batch[k]->req.wsum) dw[k] = sc.alloc<double>(nc);
    if (!dc[k] || (batch[k]->req.wsum && !dw[k])) return GS_ENOMEM;
  }
  int st = count3_batch_device(gr.data(), ng, weighted ? fws.data() : nullptr, dc.data(), dw.data(),
                               o, sc);
  for (int k = 0; k < ng && !st; ++k) {
    st = cuda_status(cudaMemcpyAsync(batch[k]->req.counts, dc[k], sizeof(uint64_t) * nc,
                                     cudaMemcpyDeviceToHost, o.stream));
    if (!st && dw[k])
      st = cuda_status(cudaMemcpyAsync(batch[k]->req.wsum, dw[k], sizeof(double) * nc,
                                       cudaMemcpyDeviceToHost, o.stream));
  }
  cudaError_t e = cudaStreamSynchronize(o.stream);
  return st ? st : cuda_status(e);
}

int run_4pcf(gs_server* S, const std::shared_ptr<Job>& j) {
  gs_options o{};
  o.stream = S->s_count;
  return gs_count_4pcf_parity(j->graph, j->w.empty() ? nullptr : j->w.data(), j->req.counts,
                              j->req.odd, j->req.wsum, nullptr, &o);
}

void counter_loop(gs_server* S) {
  cudaSetDevice(S->device);
  for (;;) {
    std::vector<std::shared_ptr<Job>> take;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv_ready.wait(lk, [&] { return S->stop || !S->ready.empty(); });
      if (S->stop && S->ready.empty()) return;
      while (!S->ready.empty()) {
        take.push_back(S->ready.front());
        S->ready.pop_front();
      }
    }
    // group 3pCF requests by (nb, weighted); batches of at most max_batch
    std::map<std::pair<int, bool>, std::vector<std::shared_ptr<Job>>> groups;
    for (auto& j : take) {
      if (j->req.npoint == 4) {
        finish(S, j, run_4pcf(S, j));
        continue;
      }
      groups[{j->req.nb, !j->w.empty()}].push_back(j);
    }
    for (auto& kv : groups) {
      auto& v = kv.second;
      for (size_t b = 0; b < v.size(); b += (size_t)S->cfg.max_batch) {
        std::vector<std::shared_ptr<Job>> batch(
            v.begin() + b, v.begin() + std::min(v.size(), b + (size_t)S->cfg.max_batch));
        const int st = run_3pcf_batch(S, batch);
        for (auto& j : batch) finish(S, j, st);
      }
    }
  }
}

}  // namespace
}  // namespace gs

using namespace gs;

extern "C" {

int gs_server_create(const gs_server_config* cfg, gs_server** out) {
  if (!out) return GS_EINVAL;
  *out = nullptr;
  gs_server* S = new (std::nothrow) gs_server();
  if (!S) return GS_ENOMEM;
  if (cfg) S->cfg = *cfg;
  if (S->cfg.max_batch <= 0) S->cfg.max_batch = 64;
  cudaGetDevice(&S->device);
  if (S->cfg.device_budget_bytes == 0) {
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    S->cfg.device_budget_bytes = (uint64_t)(0.8 * (double)fr);
  }
  cudaError_t e = cudaStreamCreateWithFlags(&S->s_build, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&S->s_count, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    if (S->s_build) cudaStreamDestroy(S->s_build);
    delete S;
    return cuda_status(e);
  }
  S->t0 = std::chrono::steady_clock::now();
  S->builder = std::thread(builder_loop, S);
  S->counter = std::thread(counter_loop, S);
  *out = S;
  return GS_OK;
}

int gs_server_submit(gs_server* S, const gs_request* r, int64_t* ticket) {
  if (!S || !r || !ticket || !r->edges_u || !r->counts || r->nb < 1 || r->n < 0) return GS_EINVAL;
  if ((r->npoint != 3 && r->npoint != 4) || (r->n > 0 && !r->xyz)) return GS_EINVAL;
  if (r->npoint == 4 && !r->odd) return GS_EINVAL;
  auto j = std::make_shared<Job>();
  j->req = *r;
  // inputs are copied: the caller's arrays are not retained
  j->xyz.assign(r->xyz, r->xyz + 3 * r->n);
  j->edges.assign(r->edges_u, r->edges_u + r->nb + 1);
  if (r->w) j->w.assign(r->w, r->w + r->n);
  j->req.xyz = nullptr;
  j->req.edges_u = j->edges.data();
  j->req.w = nullptr;
  std::lock_guard<std::mutex> lk(S->mu);
  if (S->stop) return GS_EINVAL;
  j->ticket = S->next_ticket++;
  j->t_submit = now_s(S->t0);
  S->jobs[j->ticket] = j;
  S->pending.push_back(j);
  S->in_flight += 1;
  *ticket = j->ticket;
  S->cv_pending.notify_all();
  return GS_OK;
}

int gs_server_wait(gs_server* S, int64_t ticket, double timeout_s, gs_ticket_info* info) {
  if (!S) return GS_EINVAL;
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->jobs.find(ticket);
  if (it == S->jobs.end()) return GS_EINVAL;
  std::shared_ptr<Job> j = it->second;
  auto pred = [&] { return j->done; };
  if (timeout_s < 0) {
    S->cv_done.wait(lk, pred);
  } else if (!S->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), pred)) {
    return GS_ETIMEOUT;
  }
  if (info) {
    info->status = j->status;
    info->t_submit = j->t_submit;
    info->t_start = j->t_start;
    info->t_done = j->t_done;
  }
  S->jobs.erase(it);
  return j->status;
}

int gs_server_destroy(gs_server* S) {
  if (!S) return GS_OK;
  {
    // let queued requests finish first
    std::unique_lock<std::mutex> lk(S->mu);
    S->cv_done.wait(lk, [&] { return S->in_flight == 0; });
    S->stop = true;
    S->cv_pending.notify_all();
    S->cv_ready.notify_all();
    S->cv_mem.notify_all();
  }
  S->builder.join();
  S->counter.join();
  cudaStreamDestroy(S->s_build);
  cudaStreamDestroy(S->s_count);
  delete S;
  return GS_OK;
}

}  // extern "C"
