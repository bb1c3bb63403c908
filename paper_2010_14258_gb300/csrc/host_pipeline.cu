// ldbp_apply on host-resident waveforms: chunked copy-in / compute /
// copy-out on library streams (one in, two compute, one out), so that the
// host <-> device transfers of one group of waveforms overlap the fused LDBP
// pass of another, and consecutive passes overlap each other's last wave.
#include <cstring>
#include <mutex>

#include "common.cuh"

namespace ldbp {

namespace {

constexpr int kMaxDev = 64;
constexpr int kMaxChunks = 256;

// Library-owned streams and events, created once per device.
struct PipeStreams {
  cudaStream_t in = nullptr, cmp[2] = {nullptr, nullptr}, out = nullptr;
  cudaEvent_t start = nullptr, join[4] = {};
  cudaEvent_t ev_in[kMaxChunks] = {}, ev_cmp[kMaxChunks] = {};
  bool ready = false;
};

PipeStreams g_pipes[kMaxDev];
std::mutex g_pipe_mu;

cudaError_t pipe_streams(int dev, PipeStreams** out) {
  if (dev < 0 || dev >= kMaxDev) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_pipe_mu);
  PipeStreams& ps = g_pipes[dev];
  if (!ps.ready) {
    cudaError_t e = cudaStreamCreateWithFlags(&ps.in, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ps.cmp[0], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ps.cmp[1], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ps.out, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ps.start, cudaEventDisableTiming);
    for (int i = 0; i < 4 && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&ps.join[i], cudaEventDisableTiming);
    for (int i = 0; i < kMaxChunks && e == cudaSuccess; ++i) {
      e = cudaEventCreateWithFlags(&ps.ev_in[i], cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ps.ev_cmp[i], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) return e;
    ps.ready = true;
  }
  *out = &ps;
  return cudaSuccess;
}

// Enqueues every chunk: copy-in on `in`, the pass on one of the two compute
// streams, copy-out on `out`, ordered by events.
int enqueue_chunks(PipeStreams* ps, const void* taps, int32_t taps_stride, const int32_t* T, const float* c, int32_t M,
                   const char* xh, char* yh, char* xd, char* yd, int64_t n, int32_t batch, int32_t chunks, size_t row) {
  for (int i = 0; i < chunks; ++i) {
    const long long a = (long long)batch * i / chunks, b = (long long)batch * (i + 1) / chunks;
    if (b <= a) continue;
    const size_t off = row * (size_t)a, len = row * (size_t)(b - a);
    LDBP_CUDA_TRY(cudaMemcpyAsync(xd + off, xh + off, len, cudaMemcpyHostToDevice, ps->in));
    LDBP_CUDA_TRY(cudaEventRecord(ps->ev_in[i], ps->in));
    cudaStream_t cs = ps->cmp[i & 1];  // two compute streams: a chunk's last wave overlaps the next chunk
    LDBP_CUDA_TRY(cudaStreamWaitEvent(cs, ps->ev_in[i], 0));
    if (int rc = ldbp_apply(taps, taps_stride, T, c, M, xd + off, yd + off, n, (int32_t)(b - a), nullptr, cs))
      return rc;
    LDBP_CUDA_TRY(cudaEventRecord(ps->ev_cmp[i], cs));
    LDBP_CUDA_TRY(cudaStreamWaitEvent(ps->out, ps->ev_cmp[i], 0));
    LDBP_CUDA_TRY(cudaMemcpyAsync(yh + off, yd + off, len, cudaMemcpyDeviceToHost, ps->out));
  }
  return LDBP_OK;
}

}  // namespace
}  // namespace ldbp

using namespace ldbp;

extern "C" {

size_t ldbp_apply_host_workspace(int64_t n, int32_t batch) {
  if (n < 1 || batch < 1) return 0;
  return 2 * (size_t)n * (size_t)batch * sizeof(float2);
}

int ldbp_apply_host(const void* taps, int32_t taps_stride, const int32_t* T, const float* c, int32_t M,
                    const void* x_host, void* y_host, int64_t n, int32_t batch, int32_t chunks, void* workspace,
                    size_t workspace_bytes, void* stream) {
  if (!x_host || !y_host) return fail(LDBP_EINVAL, "x_host and y_host must be non-NULL");
  if (n < 1 || batch < 1) return fail(LDBP_EINVAL, "n=%lld, batch=%d must be >= 1", (long long)n, batch);
  if (chunks < 1 || chunks > batch || chunks > kMaxChunks)
    return fail(LDBP_EINVAL, "chunks=%d outside 1..min(batch, %d)", chunks, kMaxChunks);
  const size_t row = (size_t)n * sizeof(float2), bytes = row * (size_t)batch;
  if (!workspace || workspace_bytes < 2 * bytes)
    return fail(LDBP_EINVAL, "workspace of %zu bytes, need %zu", workspace_bytes, 2 * bytes);
  if (!aligned16(workspace)) return fail(LDBP_EINVAL, "workspace must be 16-byte aligned");
  const char* xh = static_cast<const char*>(x_host);
  char* yh = static_cast<char*>(y_host);
  if (xh < yh + bytes && yh < xh + bytes) return fail(LDBP_EINVAL, "x_host and y_host overlap");
  int dev = 0;
  LDBP_CUDA_TRY(cudaGetDevice(&dev));
  PipeStreams* ps = nullptr;
  LDBP_CUDA_TRY(pipe_streams(dev, &ps));
  std::lock_guard<std::mutex> lk(g_pipe_mu);  // one pipelined call per device at a time
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  char* xd = static_cast<char*>(workspace);
  char* yd = xd + bytes;
  LDBP_CUDA_TRY(cudaEventRecord(ps->start, st));
  LDBP_CUDA_TRY(cudaStreamWaitEvent(ps->in, ps->start, 0));
  LDBP_CUDA_TRY(cudaStreamWaitEvent(ps->cmp[0], ps->start, 0));
  LDBP_CUDA_TRY(cudaStreamWaitEvent(ps->cmp[1], ps->start, 0));
  LDBP_CUDA_TRY(cudaStreamWaitEvent(ps->out, ps->start, 0));
  const int rc = enqueue_chunks(ps, taps, taps_stride, T, c, M, xh, yh, xd, yd, n, batch, chunks, row);
  // The caller's stream waits for all four library streams, also after a
  // failure part-way, so no copy of an already enqueued chunk outlives the
  // call's place in the caller's stream order.
  cudaStream_t lib_streams[4] = {ps->in, ps->cmp[0], ps->cmp[1], ps->out};
  cudaError_t je = cudaSuccess;
  for (int i = 0; i < 4; ++i) {
    cudaError_t e = cudaEventRecord(ps->join[i], lib_streams[i]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ps->join[i], 0);
    if (e != cudaSuccess && je == cudaSuccess) je = e;
  }
  if (rc != LDBP_OK) return rc;
  if (je != cudaSuccess) return cuda_fail(je, "joining the pipeline streams");
  return LDBP_OK;
}

}  // extern "C"
