// Request loop over a resident index: continuous batching of queries with
// mixed view counts.
//
// A dispatcher thread owns `slots` batch slots; each slot has its own CUDA
// stream, pinned host staging and device buffers sized for one batch. While a
// slot is free and requests are queued, the dispatcher forms a batch from the
// head of the FIFO (up to max_batch_queries queries and max_batch_views views)
// and launches it on the slot's stream: copy in, gift_query (F-IF), optionally
// gift_rerank (S-IF), copy out, record an event. Batches of different slots
// run concurrently on the device. A batch is admitted only while the device
// bytes of all in-flight batches (slot buffers plus the per-call scratch
// estimate) stay within the memory budget. Completed events are polled; each
// request records its latency from submission to completion.
#include <chrono>
#include <cstring>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>

#include "gift_internal.cuh"

namespace gift {

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  int64_t ticket = 0;
  std::vector<float> feats;
  int32_t nv = 0;
  Clock::time_point t_submit, t_done;
  std::vector<int32_t> ids;
  std::vector<float> scores;
  bool done = false;
  gift_status st = GIFT_OK;
  std::string err;
};

struct Slot {
  cudaStream_t stream = nullptr;
  cudaEvent_t ev = nullptr;
  float* h_q = nullptr;
  float* d_q = nullptr;
  int32_t* d_ids = nullptr;
  float* d_sc = nullptr;
  int32_t* d_rids = nullptr;
  float* d_rsp = nullptr;
  int32_t* h_ids = nullptr;
  float* h_sc = nullptr;
  std::vector<std::shared_ptr<Request>> reqs;
  bool busy = false;
  size_t reserved = 0;  // admitted device bytes of the batch in flight
};

}  // namespace

struct Server {
  Index* ix = nullptr;
  gift_server_params prm{};
  int device = 0;
  size_t slot_bytes = 0;
  size_t budget = 0;
  size_t in_flight = 0;
  std::vector<Slot> slots;
  std::thread th;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<std::shared_ptr<Request>> queue;
  std::unordered_map<int64_t, std::shared_ptr<Request>> reqs;
  int64_t next_ticket = 1;
  bool stop = false;
  bool paused = false;
  std::vector<float> lat_ms;
  int64_t batches = 0, batched_queries = 0, completed = 0, failed = 0;
  int64_t admission_waits = 0;  // dispatcher passes that held a batch back for memory
  size_t peak_in_flight = 0;    // largest admitted bytes of the batches in flight at once
  size_t max_batch_bytes = 0;   // estimate for a batch of the configured maximum size
  Clock::time_point t_first, t_last;
  bool any = false;
  std::string fatal;

  // device bytes one batch of B queries and V views takes from the per-call pool
  size_t call_bytes(int64_t B, int64_t V) const {
    const int64_t D = ix->prm.dim, N = ix->prm.n_shapes, ma = ix->prm.query_ma;
    const int64_t slots_n = V * ma;
    size_t b = 0;
    b += (size_t)V * D * 2 * 2 + (size_t)(std::min<int64_t>(V, 131072) + 128) * D * 2 * 2;  // split rows
    b += (size_t)(slots_n + 128) * D * 2 * 2;                                                   // slot rows
    b += (size_t)slots_n * std::max(1, ix->max_runs) * 4;                                       // run table
    b += (size_t)B * N * (4 + 8 + 4 + 8) + (size_t)B * 4096 * 16;                               // scores, re-rank
    b += (size_t)slots_n * 64 + (size_t)V * 64 + (size_t)ix->prm.n_codewords * 64 + (64u << 20);
    return b;
  }

  void fail_batch(Slot& s, gift_status st, const std::string& msg) {
    for (auto& r : s.reqs) {
      r->st = st;
      r->err = msg;
      r->done = true;
      r->t_done = Clock::now();
      ++failed;
    }
    s.reqs.clear();
    s.busy = false;
    in_flight -= s.reserved;
    s.reserved = 0;
  }

  // launch the batch held by slot s (outside the lock)
  gift_status launch(Slot& s, std::string& msg) {
    const int D = ix->prm.dim;
    std::vector<int32_t> off(1, 0);
    for (auto& r : s.reqs) {
      std::memcpy(s.h_q + (size_t)off.back() * D, r->feats.data(), (size_t)r->nv * D * 4);
      off.push_back(off.back() + r->nv);
    }
    const int32_t B = (int32_t)s.reqs.size();
    const int32_t K = prm.topk;
    if (cudaMemcpyAsync(s.d_q, s.h_q, (size_t)off.back() * D * 4, cudaMemcpyHostToDevice, s.stream) != cudaSuccess) {
      msg = cudaGetErrorString(cudaGetLastError());
      return GIFT_ECUDA;
    }
    gift_index* h = reinterpret_cast<gift_index*>(ix);
    gift_status st = gift_query(h, s.d_q, off.data(), B, GIFT_MATCH_FIF, K, s.d_ids, s.d_sc, s.stream);
    if (st != GIFT_OK) {
      msg = gift_last_error();
      return st;
    }
    const int32_t* oid = s.d_ids;
    const float* osc = s.d_sc;
    if (prm.rerank) {
      const int32_t k1 = std::min(ix->k1, K);
      st = gift_rerank(h, s.d_ids, s.d_sc, B, K, k1, K, s.d_rids, s.d_rsp, s.stream);
      if (st != GIFT_OK) {
        msg = gift_last_error();
        return st;
      }
      oid = s.d_rids;
      osc = s.d_rsp;
    }
    if (cudaMemcpyAsync(s.h_ids, oid, (size_t)B * K * 4, cudaMemcpyDeviceToHost, s.stream) != cudaSuccess ||
        cudaMemcpyAsync(s.h_sc, osc, (size_t)B * K * 4, cudaMemcpyDeviceToHost, s.stream) != cudaSuccess ||
        cudaEventRecord(s.ev, s.stream) != cudaSuccess) {
      msg = cudaGetErrorString(cudaGetLastError());
      return GIFT_ECUDA;
    }
    return GIFT_OK;
  }

  void finish(Slot& s) {  // called with the lock held
    const int32_t K = prm.topk;
    const auto now = Clock::now();
    for (size_t b = 0; b < s.reqs.size(); ++b) {
      auto& r = s.reqs[b];
      r->ids.assign(s.h_ids + b * K, s.h_ids + (b + 1) * K);
      r->scores.assign(s.h_sc + b * K, s.h_sc + (b + 1) * K);
      r->t_done = now;
      r->done = true;
      lat_ms.push_back(std::chrono::duration<float, std::milli>(now - r->t_submit).count());
      if (!any) {
        t_first = r->t_submit;
        any = true;
      }
      t_last = now;
      ++completed;
    }
    s.reqs.clear();
    s.busy = false;
    in_flight -= s.reserved;
    s.reserved = 0;
  }

  void run() {
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lk(mu);
    for (;;) {
      bool progressed = false;
      // completions
      for (auto& s : slots) {
        if (!s.busy) continue;
        const cudaError_t e = cudaEventQuery(s.ev);
        if (e == cudaSuccess) {
          finish(s);
          progressed = true;
        } else if (e != cudaErrorNotReady) {
          cudaGetLastError();
          fail_batch(s, GIFT_ECUDA, cudaGetErrorString(e));
          progressed = true;
        }
      }
      if (progressed) cv_done.notify_all();
      bool busy_any = false;
      for (auto& s : slots) busy_any |= s.busy;
      if (stop && queue.empty() && !busy_any) break;
      // admissions
      for (auto& s : slots) {
        if (s.busy || queue.empty() || paused) continue;
        int64_t views = 0;
        std::vector<std::shared_ptr<Request>> take;
        while (!queue.empty() && (int32_t)take.size() < prm.max_batch_queries &&
               views + queue.front()->nv <= prm.max_batch_views) {
          views += queue.front()->nv;
          take.push_back(queue.front());
          queue.pop_front();
        }
        if (take.empty()) continue;
        const size_t need = call_bytes((int64_t)take.size(), views);
        if (in_flight > 0 && in_flight + need > budget) {  // wait for memory to free up
          for (auto it = take.rbegin(); it != take.rend(); ++it) queue.push_front(*it);
          ++admission_waits;
          break;
        }
        s.reqs = std::move(take);
        s.busy = true;
        s.reserved = need;
        in_flight += need;
        peak_in_flight = std::max(peak_in_flight, in_flight);
        ++batches;
        batched_queries += (int64_t)s.reqs.size();
        lk.unlock();
        std::string msg;
        const gift_status st = launch(s, msg);
        lk.lock();
        if (st != GIFT_OK) {
          fail_batch(s, st, msg);
          cv_done.notify_all();
        }
        progressed = true;
      }
      if (!progressed) cv_work.wait_for(lk, std::chrono::microseconds(50));
    }
  }
};

}  // namespace gift

using gift::Server;

extern "C" {

gift_status gift_server_create(gift_index* index, const gift_server_params* params, gift_server** out) {
  return gift::guarded("gift_server_create", [&] {
    GIFT_REQUIRE(index && params && out, "NULL argument");
    const gift_server_params p = *params;
    GIFT_REQUIRE(p.slots >= 1 && p.slots <= 16, "slots must be in [1, 16]");
    GIFT_REQUIRE(p.max_batch_queries >= 1 && p.max_batch_views >= 1, "batch limits must be positive");
    GIFT_REQUIRE(p.topk >= 1 && p.topk <= 1024, "topk must be in [1, 1024]");
    std::unique_ptr<Server> sv(new Server());
    sv->ix = reinterpret_cast<gift::Index*>(index);
    if (!sv->ix->ready()) gift::fail(GIFT_ESTATE, "the streamed build of this index is not complete");
    GIFT_REQUIRE(!p.rerank || sv->ix->sif_off, "re-ranking needs an index with an S-IF");
    if (sv->ix->prm.rescore_r > 0)
      GIFT_REQUIRE(p.topk <= std::min(sv->ix->prm.rescore_r, sv->ix->prm.n_shapes), "topk exceeds the rescore depth");
    sv->prm = p;
    sv->paused = p.start_paused != 0;
    GIFT_CUDA(cudaGetDevice(&sv->device));
    const int D = sv->ix->prm.dim;
    const size_t Bq = p.max_batch_queries, V = p.max_batch_views, K = p.topk;
    sv->slot_bytes = V * D * 4 + Bq * K * 16;
    size_t free_b = 0, total_b = 0;
    GIFT_CUDA(cudaMemGetInfo(&free_b, &total_b));
    sv->max_batch_bytes = sv->call_bytes((int64_t)Bq, (int64_t)V);
    const size_t per_batch = sv->slot_bytes + sv->max_batch_bytes;
    sv->budget = p.memory_budget > 0 ? (size_t)p.memory_budget : (size_t)(0.8 * (double)free_b);
    GIFT_REQUIRE(sv->slot_bytes * p.slots + per_batch <= sv->budget,
                 "memory budget too small for one batch of the configured size");
    sv->in_flight = 0;
    sv->slots.resize(p.slots);
    for (auto& s : sv->slots) {
      GIFT_CUDA(cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking));
      GIFT_CUDA(cudaEventCreateWithFlags(&s.ev, cudaEventDisableTiming));
      GIFT_CUDA(cudaMallocHost(&s.h_q, V * D * 4));
      GIFT_CUDA(cudaMalloc(&s.d_q, V * D * 4));
      GIFT_CUDA(cudaMalloc(&s.d_ids, Bq * K * 4));
      GIFT_CUDA(cudaMalloc(&s.d_sc, Bq * K * 4));
      GIFT_CUDA(cudaMalloc(&s.d_rids, Bq * K * 4));
      GIFT_CUDA(cudaMalloc(&s.d_rsp, Bq * K * 4));
      GIFT_CUDA(cudaMallocHost(&s.h_ids, Bq * K * 4));
      GIFT_CUDA(cudaMallocHost(&s.h_sc, Bq * K * 4));
    }
    sv->budget -= sv->slot_bytes * p.slots;  // what is left for the per-call scratch of in-flight batches
    Server* raw = sv.get();
    sv->th = std::thread([raw] { raw->run(); });
    *out = reinterpret_cast<gift_server*>(sv.release());
  });
}

gift_status gift_server_submit(gift_server* server, const float* q_feats, int32_t n_views, int64_t* ticket) {
  return gift::guarded("gift_server_submit", [&] {
    GIFT_REQUIRE(server && q_feats && ticket, "NULL argument");
    Server& sv = *reinterpret_cast<Server*>(server);
    GIFT_REQUIRE(n_views >= 1 && n_views <= sv.prm.max_batch_views, "view count outside [1, max_batch_views]");
    auto r = std::make_shared<gift::Request>();
    r->feats.assign(q_feats, q_feats + (size_t)n_views * sv.ix->prm.dim);
    r->nv = n_views;
    {
      std::lock_guard<std::mutex> lk(sv.mu);
      if (sv.stop) gift::fail(GIFT_ESTATE, "server is shutting down");
      r->ticket = sv.next_ticket++;
      r->t_submit = gift::Clock::now();
      sv.reqs[r->ticket] = r;
      sv.queue.push_back(r);
      *ticket = r->ticket;
    }
    sv.cv_work.notify_one();
  });
}

gift_status gift_server_wait(gift_server* server, int64_t ticket, int32_t timeout_ms, int32_t* out_ids,
                             float* out_scores) {
  return gift::guarded("gift_server_wait", [&] {
    GIFT_REQUIRE(server, "NULL server");
    Server& sv = *reinterpret_cast<Server*>(server);
    std::unique_lock<std::mutex> lk(sv.mu);
    auto it = sv.reqs.find(ticket);
    if (it == sv.reqs.end()) gift::fail(GIFT_EINVAL, "unknown ticket");
    std::shared_ptr<gift::Request> r = it->second;
    const bool ok = sv.cv_done.wait_for(lk, std::chrono::milliseconds(std::max(0, timeout_ms)), [&] { return r->done; });
    if (!ok) gift::fail(GIFT_ETIMEOUT, "request not complete within the timeout");
    sv.reqs.erase(ticket);
    if (r->st != GIFT_OK) gift::fail(r->st, r->err);
    if (out_ids) std::copy(r->ids.begin(), r->ids.end(), out_ids);
    if (out_scores) std::copy(r->scores.begin(), r->scores.end(), out_scores);
  });
}

gift_status gift_server_resume(gift_server* server) {
  return gift::guarded("gift_server_resume", [&] {
    GIFT_REQUIRE(server, "NULL server");
    Server& sv = *reinterpret_cast<Server*>(server);
    {
      std::lock_guard<std::mutex> lk(sv.mu);
      sv.paused = false;
    }
    sv.cv_work.notify_one();
  });
}

gift_status gift_server_stats(gift_server* server, gift_server_stats_t* out) {
  return gift::guarded("gift_server_stats", [&] {
    GIFT_REQUIRE(server && out, "NULL argument");
    Server& sv = *reinterpret_cast<Server*>(server);
    std::lock_guard<std::mutex> lk(sv.mu);
    gift_server_stats_t t{};
    t.completed = sv.completed;
    t.failed = sv.failed;
    t.batches = sv.batches;
    t.mean_batch = sv.batches ? (float)sv.batched_queries / (float)sv.batches : 0.f;
    t.queued = (int64_t)sv.queue.size();
    t.admission_waits = sv.admission_waits;
    t.peak_in_flight_bytes = (int64_t)sv.peak_in_flight;
    t.budget_bytes = (int64_t)sv.budget;
    t.max_batch_bytes = (int64_t)sv.max_batch_bytes;
    t.slot_bytes = (int64_t)(sv.slot_bytes * sv.slots.size());
    if (!sv.lat_ms.empty()) {
      std::vector<float> v = sv.lat_ms;
      auto pct = [&](double q) {
        const size_t i = std::min(v.size() - 1, (size_t)(q * (double)(v.size() - 1) + 0.5));
        std::nth_element(v.begin(), v.begin() + i, v.end());
        return v[i];
      };
      t.p50_ms = pct(0.50);
      t.p99_ms = pct(0.99);
      float mx = 0.f;
      for (float x : sv.lat_ms) mx = std::max(mx, x);
      t.max_ms = mx;
      const double span = std::chrono::duration<double>(sv.t_last - sv.t_first).count();
      t.queries_per_s = span > 0 ? (float)((double)sv.completed / span) : 0.f;
    }
    *out = t;
  });
}

void gift_server_destroy(gift_server* server) {
  if (!server) return;
  Server* sv = reinterpret_cast<Server*>(server);
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
    sv->paused = false;
  }
  sv->cv_work.notify_all();
  if (sv->th.joinable()) sv->th.join();
  for (auto& s : sv->slots) {
    if (s.stream) cudaStreamSynchronize(s.stream);
    cudaFreeHost(s.h_q);
    cudaFree(s.d_q);
    cudaFree(s.d_ids);
    cudaFree(s.d_sc);
    cudaFree(s.d_rids);
    cudaFree(s.d_rsp);
    cudaFreeHost(s.h_ids);
    cudaFreeHost(s.h_sc);
    if (s.ev) cudaEventDestroy(s.ev);
    if (s.stream) cudaStreamDestroy(s.stream);
  }
  delete sv;
}

}  // extern "C"
