// The diffeomorphic sampler of Sec. 3.3: a background thread keeps a bounded
// concurrent bucket of morphed samples filled (base samples drawn on the
// device, pushed through pdmp_morph, copied to pinned host memory), while the
// planner's thread draws from the bucket without ever blocking on the GPU;
// when the bucket is empty it draws from the prior instead, so a slow or
// failed GPU only reverts the planner to its plain sampling distribution.
//
// Base samples come from a counter-based generator (Philox4x32 with 10
// rounds, Salmon et al., SC'11): coordinate j of sample i of batch b is word
// (i d + j) mod 4 of block (i d + j) / 4 under counter (block, b) and key
// (seed), mapped to the box by its top 24 bits.  The prior on the host uses
// the same generator under a different key.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <mutex>
#include <thread>
#include <vector>

#include "kernels.cuh"

namespace pdmp {

__host__ __device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
  for (int r = 0; r < 10; ++r) {
    const uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
    const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c[1] ^ k0;
    const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c[3] ^ k1;
    c[1] = (uint32_t)p1;
    c[3] = (uint32_t)p0;
    c[0] = n0;
    c[2] = n2;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
}

struct SamplerBox {
  float lo[8], hi[8];
  int d;
};

__host__ __device__ __forceinline__ float box_coord(uint32_t word, float lo, float hi) {
  const float u = (float)(word >> 8) * (1.0f / 16777216.0f);
  return fmaf(u, hi - lo, lo);
}

// one thread per Philox block of 4 coordinates
__global__ void k_uniform_batch(uint64_t seed, uint64_t batch, int64_t n, SamplerBox box, float* __restrict__ x) {
  const int64_t total = n * box.d;
  const int64_t blk = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (blk * 4 >= total) return;
  uint32_t c[4] = {(uint32_t)blk, (uint32_t)((uint64_t)blk >> 32), (uint32_t)batch, (uint32_t)(batch >> 32)};
  philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
  for (int w = 0; w < 4; ++w) {
    const int64_t e = blk * 4 + w;
    if (e < total) {
      const int j = (int)(e % box.d);
      x[e] = box_coord(c[w], box.lo[j], box.hi[j]);
    }
  }
}

}  // namespace pdmp

using namespace pdmp_host;

// ------------------------------------------------------------------ queue
struct pdmp_queue {
  int d = 0;
  int64_t cap = 0;        // samples
  std::vector<float> buf; // cap x d ring
  int64_t head = 0;       // oldest sample
  int64_t count = 0;
  bool closed = false;
  std::mutex mu;
  std::condition_variable not_full;
};

extern "C" {

pdmp_status pdmp_queue_create(int32_t d, int64_t capacity, pdmp_queue** out) {
  if (out == nullptr || d < 1 || d > 8 || capacity < 1 || capacity > ((int64_t)1 << 34) / d) return PDMP_ERR_INVALID_ARG;
  pdmp_queue* q = new (std::nothrow) pdmp_queue();
  if (q == nullptr) return PDMP_ERR_INVALID_ARG;
  q->d = d;
  q->cap = capacity;
  try {
    q->buf.resize((size_t)capacity * d);
  } catch (...) {
    delete q;
    return PDMP_ERR_INVALID_ARG;
  }
  *out = q;
  return PDMP_OK;
}

pdmp_status pdmp_queue_push(pdmp_queue* q, const float* x, int64_t n, int32_t timeout_ms, int64_t* pushed) {
  if (q == nullptr || n < 0 || (n > 0 && x == nullptr) || timeout_ms < 0) return PDMP_ERR_INVALID_ARG;
  const auto deadline = std::chrono::steady_clock::now() + std::chrono::milliseconds(timeout_ms);
  int64_t done = 0;
  std::unique_lock<std::mutex> lk(q->mu);
  while (done < n && !q->closed) {
    if (q->count == q->cap) {
      if (q->not_full.wait_until(lk, deadline) == std::cv_status::timeout && q->count == q->cap) break;
      continue;
    }
    const int64_t room = q->cap - q->count;
    const int64_t take = std::min(room, n - done);
    for (int64_t i = 0; i < take; ++i) {
      const int64_t slot = (q->head + q->count + i) % q->cap;
      std::memcpy(&q->buf[(size_t)slot * q->d], x + (size_t)(done + i) * q->d, sizeof(float) * q->d);
    }
    q->count += take;
    done += take;
  }
  if (pushed) *pushed = done;
  return PDMP_OK;
}

pdmp_status pdmp_queue_pop(pdmp_queue* q, float* out, int64_t n, int64_t* popped) {
  if (q == nullptr || n < 0 || (n > 0 && out == nullptr)) return PDMP_ERR_INVALID_ARG;
  int64_t take;
  {
    std::lock_guard<std::mutex> lk(q->mu);
    take = std::min(n, q->count);
    for (int64_t i = 0; i < take; ++i) {
      const int64_t slot = (q->head + i) % q->cap;
      std::memcpy(out + (size_t)i * q->d, &q->buf[(size_t)slot * q->d], sizeof(float) * q->d);
    }
    q->head = (q->head + take) % q->cap;
    q->count -= take;
  }
  if (take > 0) q->not_full.notify_all();
  if (popped) *popped = take;
  return PDMP_OK;
}

pdmp_status pdmp_queue_size(pdmp_queue* q, int64_t* n) {
  if (q == nullptr || n == nullptr) return PDMP_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(q->mu);
  *n = q->count;
  return PDMP_OK;
}

pdmp_status pdmp_queue_close(pdmp_queue* q) {
  if (q == nullptr) return PDMP_ERR_INVALID_ARG;
  {
    std::lock_guard<std::mutex> lk(q->mu);
    q->closed = true;
  }
  q->not_full.notify_all();
  return PDMP_OK;
}

pdmp_status pdmp_queue_destroy(pdmp_queue* q) {
  if (q == nullptr) return PDMP_ERR_INVALID_ARG;
  delete q;
  return PDMP_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ sampler
struct pdmp_sampler {
  pdmp_field field{};
  pdmp_sampler_config cfg{};
  pdmp_queue* q = nullptr;
  int device = 0;
  cudaStream_t stream = nullptr;
  float *x0 = nullptr, *xT = nullptr, *host = nullptr;
  void* ws = nullptr;
  size_t ws_bytes = 0;
  std::thread producer;
  std::atomic<bool> stop{false};
  std::atomic<int64_t> produced{0}, drawn_morphed{0}, drawn_prior{0}, batches{0};
  std::atomic<int32_t> error{0};
  std::atomic<uint64_t> prior_counter{0};
};

static void sampler_free(pdmp_sampler* s) {
  if (s->q) pdmp_queue_destroy(s->q);
  int cur = 0;
  const bool restore = cudaGetDevice(&cur) == cudaSuccess && cur != s->device;
  if (restore) cudaSetDevice(s->device);
  if (s->x0) cudaFree(s->x0);
  if (s->xT) cudaFree(s->xT);
  if (s->ws) cudaFree(s->ws);
  if (s->host) cudaFreeHost(s->host);
  if (s->stream) cudaStreamDestroy(s->stream);
  if (restore) cudaSetDevice(cur);
  delete s;
}

static void producer_loop(pdmp_sampler* s) {
  if (cudaSetDevice(s->device) != cudaSuccess) {
    s->error = PDMP_ERR_CUDA;
    return;
  }
  const pdmp_sampler_config& c = s->cfg;
  pdmp::SamplerBox box{};
  box.d = c.d;
  for (int j = 0; j < c.d; ++j) {
    box.lo[j] = c.lo[j];
    box.hi[j] = c.hi[j];
  }
  const int64_t n = c.batch;
  const unsigned blocks = (unsigned)((n * c.d + 4 * 256 - 1) / (4 * 256));
  for (uint64_t b = 0; !s->stop.load(); ++b) {
    pdmp::k_uniform_batch<<<blocks, 256, 0, s->stream>>>(c.seed, b, n, box, s->x0);
    pdmp_status st = pdmp_morph(&s->field, s->x0, n, c.T, c.eta, s->xT, nullptr, 0, s->ws, s->ws_bytes, s->stream);
    if (st == PDMP_OK &&
        cudaMemcpyAsync(s->host, s->xT, sizeof(float) * n * c.d, cudaMemcpyDeviceToHost, s->stream) != cudaSuccess)
      st = PDMP_ERR_CUDA;
    if (st == PDMP_OK && cudaStreamSynchronize(s->stream) != cudaSuccess) st = PDMP_ERR_CUDA;
    if (st != PDMP_OK) {
      s->error = st;
      return;
    }
    int64_t done = 0;
    while (done < n && !s->stop.load()) {
      int64_t pushed = 0;
      pdmp_queue_push(s->q, s->host + (size_t)done * c.d, n - done, 50, &pushed);
      done += pushed;
    }
    s->produced += done;
    s->batches += 1;
  }
}

extern "C" {

pdmp_status pdmp_sampler_create(const pdmp_field* f, const pdmp_sampler_config* cfg, pdmp_sampler** out) {
  pdmp_status st = check_field(f);
  if (st != PDMP_OK) return st;
  if (cfg == nullptr || out == nullptr) return PDMP_ERR_INVALID_ARG;
  if (cfg->d != f->d || cfg->batch < 1 || cfg->capacity < cfg->batch || cfg->T < 0) return PDMP_ERR_INVALID_ARG;
  if ((st = check_step(f, cfg->eta)) != PDMP_OK) return st;
  for (int j = 0; j < cfg->d; ++j)
    if (!(cfg->hi[j] > cfg->lo[j]) || !std::isfinite(cfg->lo[j]) || !std::isfinite(cfg->hi[j]))
      return PDMP_ERR_INVALID_ARG;
  pdmp_sampler* s = new (std::nothrow) pdmp_sampler();
  if (s == nullptr) return PDMP_ERR_INVALID_ARG;
  s->field = *f;
  s->cfg = *cfg;
  cudaError_t e = cudaGetDevice(&s->device);
  if ((st = pdmp_queue_create(cfg->d, cfg->capacity, &s->q)) != PDMP_OK) {
    sampler_free(s);
    return st;
  }
  const size_t bytes = sizeof(float) * (size_t)cfg->batch * cfg->d;
  s->ws_bytes = pdmp_morph_workspace(f, cfg->batch);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMalloc(&s->x0, bytes);
  if (e == cudaSuccess) e = cudaMalloc(&s->xT, bytes);
  if (e == cudaSuccess && s->ws_bytes) e = cudaMalloc(&s->ws, s->ws_bytes);
  if (e == cudaSuccess) e = cudaMallocHost(&s->host, bytes);
  if (e != cudaSuccess) {
    sampler_free(s);
    return cuda_status(e);
  }
  s->producer = std::thread(producer_loop, s);
  *out = s;
  return PDMP_OK;
}

pdmp_status pdmp_sampler_draw(pdmp_sampler* s, float* out, int64_t n, int64_t* n_morphed) {
  if (s == nullptr || n < 0 || (n > 0 && out == nullptr)) return PDMP_ERR_INVALID_ARG;
  int64_t got = 0;
  pdmp_queue_pop(s->q, out, n, &got);
  // the rest from the prior: the same generator under another key, on the host
  const int d = s->cfg.d;
  const uint64_t key = s->cfg.seed ^ 0xA5A5A5A55A5A5A5Aull;
  const int64_t rest = n - got;
  if (rest > 0) {
    const uint64_t first = s->prior_counter.fetch_add((uint64_t)(rest * d + 3) / 4);
    for (int64_t e = 0; e < rest * d; e += 4) {
      uint32_t c[4] = {(uint32_t)(first + e / 4), (uint32_t)((first + e / 4) >> 32), 0u, 0u};
      pdmp::philox4x32_10(c, (uint32_t)key, (uint32_t)(key >> 32));
      for (int w = 0; w < 4 && e + w < rest * d; ++w) {
        const int j = (int)((e + w) % d);
        out[(size_t)got * d + e + w] = pdmp::box_coord(c[w], s->cfg.lo[j], s->cfg.hi[j]);
      }
    }
  }
  s->drawn_morphed += got;
  s->drawn_prior += rest;
  if (n_morphed) *n_morphed = got;
  return PDMP_OK;
}

pdmp_status pdmp_sampler_stats(pdmp_sampler* s, pdmp_sampler_stats_t* st) {
  if (s == nullptr || st == nullptr) return PDMP_ERR_INVALID_ARG;
  st->produced = s->produced.load();
  st->batches = s->batches.load();
  st->drawn_morphed = s->drawn_morphed.load();
  st->drawn_prior = s->drawn_prior.load();
  pdmp_queue_size(s->q, &st->queued);
  st->error = s->error.load();
  return PDMP_OK;
}

pdmp_status pdmp_sampler_destroy(pdmp_sampler* s) {
  if (s == nullptr) return PDMP_ERR_INVALID_ARG;
  s->stop = true;
  pdmp_queue_close(s->q);
  if (s->producer.joinable()) s->producer.join();
  sampler_free(s);
  return PDMP_OK;
}

}  // extern "C"
