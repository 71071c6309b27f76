// lcp_serve.cu -- a request loop around the codec (lcp_server_*).
//
// Producers submit compression requests (the next frame of their stream)
// and decompression requests (one of their earlier frames) as they arrive.
// The server keeps each producer's LCP-T/FSM reference state (a trajectory,
// Algorithm 1) and its recent containers on the device, admits requests
// against a device-memory budget, and runs them on lanes: host threads with
// their own context and CUDA stream, so requests of different producers
// overlap on the GPU.  A producer's requests run one at a time in arrival
// order.  Decompressing an earlier frame replays what its decoding needs
// (Sec. "Spatial-Anchor-Frame-Based Batch Compression": a frame depends on
// its batch and the batch's anchor only): from the latest LCP-S frame of its
// batch up to it, or from the batch's anchor when the batch opens with LCP-T,
// the frames before the requested one to codes only.  The frames a request
// needs are pinned from its admission to its completion, so eviction never
// takes them.  Containers live in stream-ordered device memory (a pool that
// keeps freed memory), so no request synchronizes the device to allocate.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "../../include/lcp.h"

namespace lcp {
int decode_chain(lcp_ctx *c, lcp_traj *t, const void *const *ins, const size_t *sizes, int k,
                 float *out, uint64_t n_cap, uint64_t *n_out, uint32_t *d_out, cudaStream_t s);
}

namespace {

using Clock = std::chrono::steady_clock;

struct Frame {
  uint64_t index = 0;
  void *buf = nullptr;  // container, device, exactly `size` bytes
  size_t size = 0;
  lcp_method method = LCP_SPATIAL;
  uint64_t anchor = 0;  // the anchor frame in force when this frame was coded
  bool has_anchor = false;
  int pins = 0;         // admitted requests that need this container
};

struct Pending {
  uint64_t ticket;
  lcp_request req;
  double enqueue_ms;
  std::vector<uint64_t> chain;  // decompress: the frames to decode, pinned
};

struct Producer {
  lcp_traj *traj = nullptr;  // encoder-side state
  uint64_t next = 0;         // index of the next frame to compress
  uint64_t n = 0;
  uint32_t d = 0;
  bool anchor_known = false;
  uint64_t anchor = 0;       // latest anchor frame (S, first of its batch)
  std::map<uint64_t, Frame> frames;  // retained containers
  std::deque<Pending> queue;
  bool queued = false;       // in the ready list
  bool busy = false;         // a lane is running one of its requests
};

}  // namespace

struct lcp_server {
  int device = 0;
  uint32_t batch = 10;
  uint64_t budget = 0;
  uint32_t retain = 20;
  std::vector<lcp_ctx *> ctxs;
  std::vector<cudaStream_t> streams;
  std::vector<void *> scratch;  // per lane: compress output / decode buffers
  std::vector<size_t> scratch_cap;
  std::vector<lcp_traj *> dec;  // per lane: decoder state, reused by every decompress
  std::vector<std::thread> threads;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  bool stop = false;
  Clock::time_point t0;
  uint64_t next_ticket = 1;
  uint64_t stored = 0;    // bytes of retained containers
  uint64_t reserved = 0;  // bytes promised to admitted, unfinished requests
  std::unordered_map<uint32_t, Producer> prods;
  std::deque<uint32_t> ready;
  std::unordered_map<uint64_t, lcp_response> done;
  std::unordered_set<uint64_t> outstanding;  // issued, not yet waited for
  std::unordered_map<uint64_t, uint64_t> promised;  // ticket -> reserved bytes

  double now_ms() const {
    return std::chrono::duration<double, std::milli>(Clock::now() - t0).count();
  }
  // device bytes held: workspaces, trajectories, containers, promises
  uint64_t in_use_locked() const {
    uint64_t b = stored + reserved;
    for (lcp_ctx *c : ctxs) b += lcp_ctx_device_bytes(c);
    for (size_t i = 0; i < scratch_cap.size(); ++i) b += scratch_cap[i];
    for (const auto &kv : prods) b += lcp_traj_device_bytes(kv.second.traj);
    for (lcp_traj *t : dec) b += lcp_traj_device_bytes(t);
    return b;
  }
};

namespace {

// frees containers older than the retention window, keeping the anchors the
// retained frames need and every frame an admitted request has pinned
// (stream-ordered free on the evicting lane's stream: nothing else uses an
// unpinned container)
void evict_locked(lcp_server *S, Producer &P, cudaStream_t st) {
  if (P.next <= S->retain) return;
  const uint64_t keep_from = P.next - S->retain;
  std::vector<uint64_t> anchors;  // anchors of retained frames
  for (const auto &kv : P.frames)
    if (kv.first >= keep_from && kv.second.has_anchor) anchors.push_back(kv.second.anchor);
  auto needed = [&](uint64_t g) {
    return std::find(anchors.begin(), anchors.end(), g) != anchors.end();
  };
  for (auto it = P.frames.begin(); it != P.frames.end();) {
    if (it->first < keep_from && !needed(it->first) && it->second.pins == 0) {
      cudaFreeAsync(it->second.buf, st);
      S->stored -= it->second.size;
      it = P.frames.erase(it);
    } else {
      ++it;
    }
  }
}

bool grow_scratch(lcp_server *S, int lane, size_t bytes) {
  if (S->scratch_cap[lane] >= bytes) return true;
  cudaStream_t st = S->streams[lane];
  if (S->scratch[lane]) cudaFreeAsync(S->scratch[lane], st);
  S->scratch[lane] = nullptr;
  S->scratch_cap[lane] = 0;
  if (cudaMallocAsync(&S->scratch[lane], bytes, st) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  S->scratch_cap[lane] = bytes;
  return true;
}

lcp_status run_compress(lcp_server *S, int lane, Producer &P, const lcp_request &r,
                        lcp_response &out) {
  lcp_ctx *ctx = S->ctxs[lane];
  cudaStream_t st = S->streams[lane];
  if (!P.traj) {
    lcp_status s = lcp_traj_create(ctx, S->batch, r.p ? r.p : 8, &P.traj);
    if (s != LCP_OK) return s;
  }
  const size_t cap = lcp_max_compressed_size(r.n, r.d);
  if (!grow_scratch(S, lane, cap)) return LCP_ERR_NOMEM;
  size_t size = 0;
  lcp_method chosen = LCP_SPATIAL;
  lcp_status s = lcp_compress(ctx, P.traj, r.d_fields, r.n, r.d, r.eb, r.mode, r.p ? r.p : 8,
                              LCP_AUTO, S->scratch[lane], S->scratch_cap[lane], &size, &chosen,
                              nullptr, st);
  if (s != LCP_OK) return s;
  Frame f;
  f.index = P.next;
  f.size = size;
  f.method = chosen;
  if (cudaMallocAsync(&f.buf, std::max<size_t>(size, 16), st) != cudaSuccess) {
    cudaGetLastError();
    return LCP_ERR_NOMEM;
  }
  const bool copy_out = r.d_bytes != nullptr && r.bytes_cap >= size;
  if (cudaMemcpyAsync(f.buf, S->scratch[lane], size, cudaMemcpyDeviceToDevice, st) !=
          cudaSuccess ||
      (copy_out && cudaMemcpyAsync(r.d_bytes, S->scratch[lane], size, cudaMemcpyDeviceToDevice,
                                   st) != cudaSuccess) ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    cudaGetLastError();
    cudaFreeAsync(f.buf, st);
    return LCP_ERR_CUDA;
  }
  // Algorithm 1 bookkeeping: an LCP-S frame that opens a batch is the anchor
  const bool first = (f.index % S->batch) == 0;
  if (chosen == LCP_SPATIAL && first) {
    P.anchor_known = true;
    P.anchor = f.index;
  }
  f.has_anchor = P.anchor_known;
  f.anchor = P.anchor;
  out.frame = f.index;
  out.size = size;
  out.method = chosen;
  std::lock_guard<std::mutex> lk(S->mu);
  P.frames[f.index] = f;
  S->stored += size;
  P.next += 1;
  evict_locked(S, P, st);
  return (r.d_bytes != nullptr && !copy_out) ? LCP_ERR_CAPACITY : LCP_OK;
}

// the frames decoding `frame` needs, in stream order (empty: not decodable)
std::vector<uint64_t> chain_locked(const lcp_server *S, const Producer &P, uint64_t frame) {
  std::vector<uint64_t> chain;
  auto it = P.frames.find(frame);
  if (it == P.frames.end()) return chain;  // never coded, or no longer retained
  const uint64_t b0 = frame - frame % S->batch;
  uint64_t start = frame;
  for (;; --start) {  // the latest LCP-S frame of the batch at or before `frame`
    auto jt = P.frames.find(start);
    if (jt == P.frames.end()) return {};
    if (jt->second.method == LCP_SPATIAL || start == b0) break;
  }
  const Frame &s0 = P.frames.at(start);
  if (s0.method == LCP_TEMPORAL) {  // the batch opens with LCP-T: its anchor first
    if (!s0.has_anchor || !P.frames.count(s0.anchor)) return {};
    chain.push_back(s0.anchor);
  }
  for (uint64_t g = start; g <= frame; ++g) chain.push_back(g);
  return chain;
}

lcp_status run_decompress(lcp_server *S, int lane, Producer &P, const Pending &job,
                          lcp_response &out) {
  const lcp_request &r = job.req;
  lcp_ctx *ctx = S->ctxs[lane];
  cudaStream_t st = S->streams[lane];
  std::vector<const void *> ins;
  std::vector<size_t> sizes;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    for (uint64_t g : job.chain) {
      const Frame &f = P.frames.at(g);  // pinned: still retained
      ins.push_back(f.buf);
      sizes.push_back(f.size);
    }
    const Frame &f = P.frames.at(job.chain.back());
    out.frame = f.index;
    out.size = f.size;
    out.method = f.method;
  }
  if (!S->dec[lane]) {
    lcp_status s = lcp_traj_create(ctx, S->batch, 8, &S->dec[lane]);
    if (s != LCP_OK) return s;
  }
  uint64_t n_out = 0;
  uint32_t d_out = 0;
  return (lcp_status)lcp::decode_chain(ctx, S->dec[lane], ins.data(), sizes.data(),
                                       (int)ins.size(), r.d_out, r.n_cap, &n_out, &d_out, st);
}

void lane_loop(lcp_server *S, int lane) {
  cudaSetDevice(S->device);
  for (;;) {
    uint32_t pid;
    Pending job;
    Producer *pp;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv_work.wait(lk, [&] { return S->stop || !S->ready.empty(); });
      if (S->ready.empty()) return;  // stopping and drained
      pid = S->ready.front();
      S->ready.pop_front();
      pp = &S->prods[pid];  // element addresses of an unordered_map are stable
      pp->queued = false;
      pp->busy = true;
      job = pp->queue.front();
      pp->queue.pop_front();
    }
    Producer &P = *pp;  // this lane owns the producer until busy is cleared
    lcp_response out{};
    out.enqueue_ms = job.enqueue_ms;
    out.start_ms = S->now_ms();
    out.status = job.req.op == LCP_REQ_COMPRESS ? run_compress(S, lane, P, job.req, out)
                                                : run_decompress(S, lane, P, job, out);
    out.done_ms = S->now_ms();
    {
      std::lock_guard<std::mutex> lk(S->mu);
      auto pr = S->promised.find(job.ticket);
      if (pr != S->promised.end()) {
        S->reserved -= pr->second;
        S->promised.erase(pr);
      }
      for (uint64_t g : job.chain) {  // unpin
        auto it = P.frames.find(g);
        if (it != P.frames.end()) it->second.pins -= 1;
      }
      S->done[job.ticket] = out;
      P.busy = false;
      if (!P.queue.empty() && !P.queued) {
        P.queued = true;
        S->ready.push_back(pid);
        S->cv_work.notify_one();
      }
    }
    S->cv_done.notify_all();
  }
}

}  // namespace

extern "C" {

lcp_status lcp_server_create(int device, int lanes, uint32_t batch, uint64_t hbm_budget,
                             lcp_server **out) {
  if (!out || lanes <= 0 || lanes > 64 || batch == 0) return LCP_ERR_ARG;
  *out = nullptr;
  if (cudaSetDevice(device) != cudaSuccess) {
    cudaGetLastError();
    return LCP_ERR_CUDA;
  }
  lcp_server *S = new lcp_server();
  S->device = device;
  S->batch = batch;
  S->budget = hbm_budget;
  S->retain = 2 * batch;
  S->t0 = Clock::now();
  {  // freed container memory stays in the device's default pool for reuse
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
      uint64_t keep = ~0ull;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    cudaGetLastError();
  }
  for (int k = 0; k < lanes; ++k) {
    lcp_ctx *c = nullptr;
    cudaStream_t st = nullptr;
    if (lcp_ctx_create(device, &c) != LCP_OK ||
        cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      if (c) lcp_ctx_destroy(c);
      lcp_server_destroy(S);
      return LCP_ERR_CUDA;
    }
    S->ctxs.push_back(c);
    S->streams.push_back(st);
    S->scratch.push_back(nullptr);
    S->scratch_cap.push_back(0);
    S->dec.push_back(nullptr);
  }
  for (int k = 0; k < lanes; ++k) S->threads.emplace_back(lane_loop, S, k);
  *out = S;
  return LCP_OK;
}

lcp_status lcp_server_submit(lcp_server *S, const lcp_request *r, uint64_t *ticket) {
  if (!S || !r || !ticket) return LCP_ERR_ARG;
  if (r->op != LCP_REQ_COMPRESS && r->op != LCP_REQ_DECOMPRESS) return LCP_ERR_ARG;
  if (r->op == LCP_REQ_COMPRESS && (!r->d_fields || r->d == 0 || r->d > 8)) return LCP_ERR_ARG;
  if (r->op == LCP_REQ_DECOMPRESS && !r->d_out) return LCP_ERR_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  if (S->stop) return LCP_ERR_STATE;
  Producer &P = S->prods[r->producer];
  const bool fresh = P.d == 0;  // no frame of this producer submitted yet
  if (r->op == LCP_REQ_COMPRESS && !fresh && (P.n != r->n || P.d != r->d)) return LCP_ERR_STATE;
  // admission: what the request may add to the device memory in use
  uint64_t need = 0;
  if (r->op == LCP_REQ_COMPRESS) {
    need = lcp_max_compressed_size(r->n, r->d);
    if (fresh) need += 6ull * (r->n * r->d + r->n) * 4;  // reference state
  }
  if (S->budget && S->in_use_locked() + need > S->budget) return LCP_ERR_NOMEM;
  if (r->op == LCP_REQ_COMPRESS && fresh) {
    P.n = r->n;
    P.d = r->d;
  }
  std::vector<uint64_t> chain;
  if (r->op == LCP_REQ_DECOMPRESS) {  // refused now when not decodable; else pinned
    chain = chain_locked(S, P, r->frame);
    if (chain.empty()) return LCP_ERR_STATE;
    for (uint64_t g : chain) P.frames.at(g).pins += 1;
  }
  const uint64_t t = S->next_ticket++;
  S->outstanding.insert(t);
  S->reserved += need;
  S->promised[t] = need;
  P.queue.push_back(Pending{t, *r, S->now_ms(), std::move(chain)});
  if (!P.queued && !P.busy) {
    P.queued = true;
    S->ready.push_back(r->producer);
    S->cv_work.notify_one();
  }
  *ticket = t;
  return LCP_OK;
}

lcp_status lcp_server_wait(lcp_server *S, uint64_t ticket, lcp_response *out) {
  if (!S || !out) return LCP_ERR_ARG;
  std::unique_lock<std::mutex> lk(S->mu);
  if (!S->outstanding.count(ticket)) return LCP_ERR_ARG;  // unknown, or waited for already
  S->cv_done.wait(lk, [&] { return S->done.count(ticket) != 0; });
  *out = S->done[ticket];
  S->done.erase(ticket);
  S->outstanding.erase(ticket);
  return LCP_OK;
}

lcp_status lcp_server_frames(lcp_server *S, uint32_t producer, uint64_t *first,
                             uint64_t *next) {
  if (!S || !first || !next) return LCP_ERR_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->prods.find(producer);
  if (it == S->prods.end() || it->second.frames.empty()) {
    *first = *next = it == S->prods.end() ? 0 : it->second.next;
    return LCP_OK;
  }
  const Producer &P = it->second;
  // the oldest frame whose batch, from its first frame on, is still retained
  // (frames after it are then retained too)
  auto decodable = [&](uint64_t f) {
    for (uint64_t g = f - f % S->batch; g <= f; ++g)
      if (!P.frames.count(g)) return false;
    return true;
  };
  uint64_t f = P.next > S->retain ? P.next - S->retain : 0;
  while (f < P.next && !decodable(f)) ++f;
  *first = f;
  *next = P.next;
  return LCP_OK;
}

uint64_t lcp_server_device_bytes(lcp_server *S) {
  if (!S) return 0;
  std::lock_guard<std::mutex> lk(S->mu);
  return S->in_use_locked();
}

lcp_status lcp_server_destroy(lcp_server *S) {
  if (!S) return LCP_ERR_ARG;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv_work.notify_all();
  for (auto &t : S->threads) t.join();
  cudaSetDevice(S->device);
  for (size_t k = 0; k < S->streams.size(); ++k) cudaStreamSynchronize(S->streams[k]);
  for (auto &kv : S->prods) {
    for (auto &f : kv.second.frames) cudaFree(f.second.buf);
    if (kv.second.traj) lcp_traj_destroy(kv.second.traj);
  }
  for (lcp_traj *t : S->dec)
    if (t) lcp_traj_destroy(t);
  for (size_t k = 0; k < S->ctxs.size(); ++k) {
    if (S->scratch[k]) cudaFree(S->scratch[k]);
    cudaStreamDestroy(S->streams[k]);
    lcp_ctx_destroy(S->ctxs[k]);
  }
  delete S;
  return LCP_OK;
}

}  // extern "C"
