// lcp_batch.cu -- many frames at once: lcp_compress_batch, lcp_decompress_batch.
//
// The frames of one time step of many trajectories (Algorithm 1 runs per
// trajectory) are independent.  Small frames leave most of the GPU idle, so
// lanes -- host threads, each with its own context and CUDA stream -- run
// different frames at the same time and their kernels overlap on the device.
// Jobs are handed out largest first from a shared counter.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <numeric>
#include <thread>
#include <vector>

#include "../../include/lcp.h"

namespace {

template <typename Job, typename Size, typename Run>
lcp_status run_batch(lcp_ctx *const *ctxs, int lanes, Job *jobs, int njobs, Size size, Run run) {
  if (lanes <= 0 || njobs < 0 || !ctxs || (njobs > 0 && !jobs)) return LCP_ERR_ARG;
  for (int k = 0; k < lanes; ++k)
    if (!ctxs[k]) return LCP_ERR_ARG;
  std::vector<int> order(njobs);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int b) { return size(jobs[a]) > size(jobs[b]); });
  std::atomic<int> next{0};
  auto lane_fn = [&](int lane) {
    for (;;) {
      const int i = next.fetch_add(1);
      if (i >= njobs) break;
      Job &J = jobs[order[i]];
      const auto t0 = std::chrono::steady_clock::now();
      J.status = run(lane, J);
      const auto t1 = std::chrono::steady_clock::now();
      J.ms = std::chrono::duration<float, std::milli>(t1 - t0).count();
    }
  };
  const int used = std::min(lanes, std::max(njobs, 1));
  std::vector<std::thread> threads;
  threads.reserve(used > 0 ? used - 1 : 0);
  for (int k = 1; k < used; ++k) threads.emplace_back(lane_fn, k);
  lane_fn(0);
  for (auto &t : threads) t.join();
  for (int i = 0; i < njobs; ++i)
    if (jobs[i].status != LCP_OK) return jobs[i].status;
  return LCP_OK;
}

}  // namespace

extern "C" lcp_status lcp_compress_batch(lcp_ctx *const *ctxs, void *const *streams, int lanes,
                                         lcp_compress_job *jobs, int njobs) {
  return run_batch(
      ctxs, lanes, jobs, njobs,
      [](const lcp_compress_job &J) { return J.n * (uint64_t)J.d; },
      [&](int lane, lcp_compress_job &J) {
        J.out_size = 0;
        J.chosen = LCP_SPATIAL;
        return lcp_compress(ctxs[lane], J.traj, J.d_fields, J.n, J.d, J.eb, J.mode, J.p,
                            J.method, J.d_out, J.out_cap, &J.out_size, &J.chosen, nullptr,
                            streams ? streams[lane] : nullptr);
      });
}

extern "C" lcp_status lcp_decompress_batch(lcp_ctx *const *ctxs, void *const *streams, int lanes,
                                           lcp_decompress_job *jobs, int njobs) {
  return run_batch(
      ctxs, lanes, jobs, njobs, [](const lcp_decompress_job &J) { return (uint64_t)J.in_size; },
      [&](int lane, lcp_decompress_job &J) {
        J.n_out = 0;
        J.d_fields = 0;
        return lcp_decompress(ctxs[lane], J.traj, J.d_in, J.in_size, J.d_out, J.n_cap, &J.n_out,
                              &J.d_fields, streams ? streams[lane] : nullptr);
      });
}
