// Serving: device-resident matrices, HBM-budget admission and continuous
// batching of SpMV requests onto the persistent batched kernels.  A request
// with one x vector is an item of the batched SpMV kernel; a request with
// 2..8 vectors is one item of the batched k-vector kernel, which streams the
// matrix once and gathers all its vectors' values of a column together.
//
// Threads: the caller's threads submit and wait; a scheduler thread packs
// queued requests into a launch whenever a context (stream + x/y arenas +
// directory buffers) is free and hands it to the context's own issuing
// thread, which issues its copies and kernels (so that the issuing of
// several launches overlaps); a completion thread polls each context's
// event, copies y back to the callers' buffers and wakes the waiters.
// Several contexts are in flight at once, so requests that arrive while
// others run are admitted as soon as a context frees up, and their work
// overlaps on the device.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "batch.cuh"
#include "common.cuh"

extern "C" msrep_status msrep_partition_csr(const msrep_matrix *A, msrep_partition *part,
                                            unsigned flags, void *stream);

namespace msrep {

int32_t effective_tile(int32_t tile);

using Clock = std::chrono::steady_clock;

struct Resident {
  int64_t id;
  int32_t m, n;
  int64_t nnz;
  int32_t np, tile;
  int64_t tiles;     // tile count of the plan
  void *mem;         // one device allocation for everything below
  size_t bytes;
  BatchItem item;    // pointers into mem
  int64_t refs = 0;  // queued or running requests
  bool dying = false;
};

struct Request {
  uint64_t id;
  int64_t matrix;
  int32_t k;
  const float *x;
  float *y;
  Clock::time_point t_submit;
  bool x_pinned = false, y_pinned = false;  // page-locked: DMA directly
  // page-locked and mapped: the device address of x / y, which the launch's
  // copy kernels read and write directly (no per-request copy)
  const float *x_map = nullptr;
  float *y_map = nullptr;
  bool done = false;
  msrep_status status = MSREP_OK;
  std::string error;  // why the request failed, when it did
};

struct Context {
  cudaStream_t stream = nullptr;
  cudaEvent_t done_ev = nullptr;  // end of the launch (also polled)
  // timing: launch start (before the x copies), kernels start and end
  cudaEvent_t begin_ev = nullptr, k0_ev = nullptr, k1_ev = nullptr;
  float *x_dev = nullptr, *y_dev = nullptr;    // arenas
  float *x_pin = nullptr, *y_pin = nullptr;    // pinned staging
  int64_t arena_floats = 0;
  // the launch directory (LaunchDir), built in dir_pin and copied to dir_dev
  char *dir_dev = nullptr;
  char *dir_pin = nullptr;
  size_t dir_bytes = 0;
  double *head = nullptr, *tail = nullptr;
  int64_t max_tiles = 0;
  // k-vector requests: interleaved x arena, partials (x8)
  float *xt_dev = nullptr;
  int64_t xt_floats = 0;
  double *head_k = nullptr, *tail_k = nullptr;
  bool busy = false;      // packed by the scheduler (launching or in flight)
  bool pending = false;   // packed, waiting for its issuing thread
  bool in_flight = false; // its event has been recorded for this launch
  std::vector<BatchItem> ritem;  // per request: its matrix
  std::vector<int64_t> rtiles;   // per request: the matrix's tile count
  std::vector<std::shared_ptr<Request>> reqs;  // in this launch
  std::vector<int64_t> y_off;                  // per request, floats into y arena
  double bytes = 0;                            // algorithmic bytes of the launch
  Clock::time_point t_launch;
};

}  // namespace msrep

struct msrep_server {
  msrep_serve_config cfg;
  std::mutex mu;
  std::condition_variable cv_work;   // scheduler: new request or free context
  std::condition_variable cv_done;   // waiters
  std::condition_variable cv_issue;  // issuing threads: a context was packed
  std::condition_variable cv_flight; // completion thread: a launch was issued, or stopping
  std::map<int64_t, msrep::Resident> mats;
  std::deque<std::shared_ptr<msrep::Request>> queue;
  std::unordered_map<uint64_t, std::shared_ptr<msrep::Request>> reqs;
  std::vector<msrep::Context> ctx;
  int64_t next_matrix = 1;
  uint64_t next_req = 1;
  int64_t resident = 0;
  bool stop = false, stop_issuers = false;
  std::thread scheduler, completer;
  std::vector<std::thread> issuers;  // one per context
  // statistics
  std::vector<double> lat_us;     // submit -> y in the caller's buffer
  std::vector<double> wait_us;    // submit -> packed into a launch (host)
  std::vector<double> dev_us;     // per launch: first copy -> last copy (device)
  std::vector<double> host_us;    // per launch: the scheduler issuing its copies and kernels
  double kernel_us = 0;           // sum over launches of the kernels' device time
  uint64_t submitted = 0, completed = 0, rejected = 0, launches = 0, items = 0;
  double work_bytes = 0, busy_s = 0;
  int inflight = 0;
  msrep::Clock::time_point busy_since;
};

namespace msrep {

// one copy of a launch's copy lists: n floats from src to dst, both
// device-accessible (the arenas, or mapped page-locked caller buffers)
struct CopyItem {
  const float *src;
  float *dst;
  int64_t n;
};

// The copy lists of a launch: blockIdx.y walks the items, the blocks along
// x share an item's floats (16-byte accesses where both ends allow).
__global__ void serve_copy(const CopyItem *items, int count) {
  for (int j = blockIdx.y; j < count; j += gridDim.y) {
    const CopyItem c = items[j];
    const bool vec = ((reinterpret_cast<uintptr_t>(c.src) | reinterpret_cast<uintptr_t>(c.dst)) & 15) == 0;
    const int64_t t0 = blockIdx.x * int64_t(blockDim.x) + threadIdx.x, step = int64_t(gridDim.x) * blockDim.x;
    int64_t done = 0;
    if (vec) {
      const int64_t n4 = c.n / 4;
      const float4 *s4 = reinterpret_cast<const float4 *>(c.src);
      float4 *d4 = reinterpret_cast<float4 *>(c.dst);
      for (int64_t i = t0; i < n4; i += step) d4[i] = s4[i];
      done = 4 * n4;
    }
    for (int64_t i = done + t0; i < c.n; i += step) c.dst[i] = c.src[i];
  }
}

static msrep_status launch_copies(const CopyItem *items, int count, cudaStream_t st) {
  if (count == 0) return MSREP_OK;
  serve_copy<<<dim3(32, std::min(count, 1024)), 256, 0, st>>>(items, count);
  MSREP_CUDA_TRY(cudaGetLastError());
  return MSREP_OK;
}

static void free_context(Context &c) {
  if (c.stream) cudaStreamSynchronize(c.stream);
  cudaFree(c.x_dev);
  cudaFree(c.y_dev);
  cudaFree(c.dir_dev);
  cudaFree(c.head);
  cudaFree(c.tail);
  cudaFree(c.xt_dev);
  cudaFree(c.head_k);
  cudaFree(c.tail_k);
  cudaFreeHost(c.x_pin);
  cudaFreeHost(c.y_pin);
  cudaFreeHost(c.dir_pin);
  if (c.done_ev) cudaEventDestroy(c.done_ev);
  if (c.begin_ev) cudaEventDestroy(c.begin_ev);
  if (c.k0_ev) cudaEventDestroy(c.k0_ev);
  if (c.k1_ev) cudaEventDestroy(c.k1_ev);
  if (c.stream) cudaStreamDestroy(c.stream);
  c = Context{};
}

// Per-launch directory, laid out for the launch's R requests (so that one
// copy of about 250 bytes a request carries it): the SpMV items (one-vector
// requests) with their tile offsets and x / y pointers, the copy lists
// (x in, y out), and the k-vector items with tile and unit offsets and
// their x / interleaved-x / y pointers.
struct LaunchDir {
  size_t items, toff, xs, ys, cin, cout, itk, toffk, uoffk, xin, xtp, ysk, bytes;
  explicit LaunchDir(size_t R) {
    size_t o = 0;
    auto take = [&o](size_t b) {
      const size_t at = o;
      o = (o + b + 15) & ~size_t(15);
      return at;
    };
    items = take(sizeof(BatchItem) * R);
    toff = take(sizeof(int64_t) * (R + 1));
    xs = take(sizeof(void *) * R);
    ys = take(sizeof(void *) * R);
    cin = take(sizeof(CopyItem) * R);
    cout = take(sizeof(CopyItem) * R);
    itk = take(sizeof(BatchItem) * R);
    toffk = take(sizeof(int64_t) * (R + 1));
    uoffk = take(sizeof(int64_t) * (R + 1));
    xin = take(sizeof(void *) * R);
    xtp = take(sizeof(void *) * R);
    ysk = take(sizeof(void *) * R);
    bytes = o;
  }
};

static size_t dir_size(int32_t max_items) { return LaunchDir(size_t(max_items)).bytes; }

// Launch the requests in c.reqs (the context's issuing thread, server lock
// NOT held; the matrices they name are pinned by their refs).  ritem /
// rtiles: each request's matrix and its tile count.  Mapped page-locked x
// and y are read and written by the launch's kernels directly: x of a
// one-vector request is copied into the arena by one copy kernel (the
// SpMV gathers it at random), x of a k-vector request is read by the
// interleaving kernel itself, and every mapped y is written by one copy
// kernel at the end.  Other buffers take one DMA copy each (staged through
// the pinned arenas when pageable).
static msrep_status launch_context(msrep_server *s, Context &c,
                                   const std::vector<BatchItem> &ritem,
                                   const std::vector<int64_t> &rtiles) {
  const size_t R = c.reqs.size();
  const LaunchDir L(R);
  if (L.bytes > c.dir_bytes) return fail(MSREP_ERR_INVALID_ARG, "launch directory too large");
  char *dp = c.dir_pin;
  BatchItem *it = reinterpret_cast<BatchItem *>(dp + L.items);
  int64_t *toff = reinterpret_cast<int64_t *>(dp + L.toff);
  const void **xs = reinterpret_cast<const void **>(dp + L.xs);
  void **ys = reinterpret_cast<void **>(dp + L.ys);
  CopyItem *cin = reinterpret_cast<CopyItem *>(dp + L.cin);
  CopyItem *cout = reinterpret_cast<CopyItem *>(dp + L.cout);
  BatchItem *itk = reinterpret_cast<BatchItem *>(dp + L.itk);
  int64_t *toffk = reinterpret_cast<int64_t *>(dp + L.toffk);
  int64_t *uoffk = reinterpret_cast<int64_t *>(dp + L.uoffk);
  const void **xin = reinterpret_cast<const void **>(dp + L.xin);
  void **xtp = reinterpret_cast<void **>(dp + L.xtp);
  void **ysk = reinterpret_cast<void **>(dp + L.ysk);

  int64_t xo = 0, yo = 0, xto = 0, tt = 0, ttk = 0, utk = 0;
  int n1 = 0, nk = 0, nci = 0, nco = 0;
  c.y_off.clear();
  MSREP_CUDA_TRY(cudaEventRecord(c.begin_ev, c.stream));
  for (size_t i = 0; i < R; ++i) {
    const auto &r = c.reqs[i];
    const BatchItem &bi = ritem[i];
    c.y_off.push_back(yo);
    const int64_t nx = int64_t(bi.n) * r->k;
    const size_t xb = sizeof(float) * size_t(nx);
    const float *xsrc = c.x_dev + xo;  // where the kernels read this request's x
    if (r->x_map && r->k > 1) {
      xsrc = r->x_map;
    } else if (r->x_map) {
      cin[nci++] = CopyItem{r->x_map, c.x_dev + xo, nx};
    } else if (r->x_pinned) {
      MSREP_CUDA_TRY(cudaMemcpyAsync(c.x_dev + xo, r->x, xb, cudaMemcpyHostToDevice, c.stream));
    } else {
      std::memcpy(c.x_pin + xo, r->x, xb);
      MSREP_CUDA_TRY(cudaMemcpyAsync(c.x_dev + xo, c.x_pin + xo, xb, cudaMemcpyHostToDevice, c.stream));
    }
    if (r->k == 1) {
      it[n1] = bi;
      toff[n1] = tt;
      tt += rtiles[i];
      xs[n1] = xsrc;
      ys[n1] = c.y_dev + yo;
      ++n1;
    } else {
      itk[nk] = bi;
      itk[nk].k = r->k;
      toffk[nk] = ttk;
      uoffk[nk] = utk;
      ttk += rtiles[i];
      utk += batched_k_units(rtiles[i], r->k);
      xin[nk] = xsrc;
      xtp[nk] = c.xt_dev + xto;
      ysk[nk] = c.y_dev + yo;
      xto += int64_t(bi.n) * kBatchWidth;
      ++nk;
    }
    if (r->y_map) cout[nco++] = CopyItem{c.y_dev + yo, r->y_map, int64_t(bi.m) * r->k};
    xo += nx;
    yo += int64_t(bi.m) * r->k;
  }
  toff[n1] = tt;
  toffk[nk] = ttk;
  uoffk[nk] = utk;
  const char *dd = c.dir_dev;
  MSREP_CUDA_TRY(cudaMemcpyAsync(c.dir_dev, c.dir_pin, L.bytes, cudaMemcpyHostToDevice, c.stream));
  MSREP_TRY(launch_copies(reinterpret_cast<const CopyItem *>(dd + L.cin), nci, c.stream));
  MSREP_CUDA_TRY(cudaEventRecord(c.k0_ev, c.stream));
  if (n1 > 0)
    MSREP_TRY(launch_batched(reinterpret_cast<const BatchItem *>(dd + L.items),
                             reinterpret_cast<const int64_t *>(dd + L.toff), n1, tt, MSREP_F32,
                             reinterpret_cast<const void *const *>(dd + L.xs),
                             reinterpret_cast<void *const *>(dd + L.ys), c.head, c.tail, 1.0, 0.0,
                             0, c.stream));
  if (nk > 0)
    MSREP_TRY(launch_batched_k(reinterpret_cast<const BatchItem *>(dd + L.itk),
                               reinterpret_cast<const int64_t *>(dd + L.toffk),
                               reinterpret_cast<const int64_t *>(dd + L.uoffk), nk, ttk, utk,
                               reinterpret_cast<const void *const *>(dd + L.xin),
                               reinterpret_cast<void *const *>(dd + L.xtp),
                               reinterpret_cast<void *const *>(dd + L.ysk), c.head_k, c.tail_k, 0,
                               c.stream));
  MSREP_CUDA_TRY(cudaEventRecord(c.k1_ev, c.stream));
  MSREP_TRY(launch_copies(reinterpret_cast<const CopyItem *>(dd + L.cout), nco, c.stream));
  for (size_t i = 0; i < R; ++i) {
    const auto &r = c.reqs[i];
    if (r->y_map) continue;
    const int64_t ylen = (i + 1 < R ? c.y_off[i + 1] : yo) - c.y_off[i];
    float *dst = r->y_pinned ? r->y : c.y_pin + c.y_off[i];
    MSREP_CUDA_TRY(cudaMemcpyAsync(dst, c.y_dev + c.y_off[i], sizeof(float) * ylen,
                                   cudaMemcpyDeviceToHost, c.stream));
  }
  MSREP_CUDA_TRY(cudaEventRecord(c.done_ev, c.stream));
  return MSREP_OK;
}

static void scheduler_loop(msrep_server *s) {
  cudaSetDevice(s->cfg.device);
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    s->cv_work.wait(lk, [&] {
      if (s->stop && s->queue.empty()) return true;
      if (s->queue.empty()) return false;
      for (auto &c : s->ctx)
        if (!c.busy) return true;
      return false;
    });
    if (s->stop && s->queue.empty()) return;
    Context *c = nullptr;
    for (auto &cc : s->ctx)
      if (!cc.busy) {
        c = &cc;
        break;
      }
    if (!c) continue;
    // pack requests in arrival order while the context has room; one-vector
    // requests fill the SpMV directory, the others the k-vector one
    std::vector<BatchItem> ritem;
    std::vector<int64_t> rtiles;
    int64_t xf = 0, yf = 0, xtf = 0, tt = 0, ttk = 0;
    int n1 = 0, nk = 0;
    double bytes = 0;
    c->reqs.clear();
    while (!s->queue.empty()) {
      auto r = s->queue.front();
      auto mit = s->mats.find(r->matrix);
      const Resident &R = mit->second;
      const int64_t nx = int64_t(R.n) * r->k, ny = int64_t(R.m) * r->k;
      const bool one = r->k == 1;
      const bool full =
          xf + nx > c->arena_floats || yf + ny > c->arena_floats ||
          (one ? (n1 + 1 > s->cfg.max_items || tt + R.tiles > c->max_tiles)
               : (nk + 1 > s->cfg.max_items || ttk + R.tiles > c->max_tiles ||
                  xtf + int64_t(R.n) * kBatchWidth > c->xt_floats));
      if (!c->reqs.empty() && full) break;
      s->queue.pop_front();
      c->reqs.push_back(r);
      ritem.push_back(R.item);
      rtiles.push_back(R.tiles);
      xf += nx;
      yf += ny;
      if (one) {
        ++n1;
        tt += R.tiles;
      } else {
        ++nk;
        ttk += R.tiles;
        xtf += int64_t(R.n) * kBatchWidth;
      }
      // algorithmic bytes (FP32 CSR): the matrix once per launch item, x and
      // y once per vector
      bytes += 8.0 * R.nnz + 4.0 * (R.m + 1) + double(r->k) * (4.0 * R.n + 4.0 * R.m);
    }
    c->busy = true;
    c->bytes = bytes;
    c->t_launch = Clock::now();
    for (const auto &r : c->reqs)
      s->wait_us.push_back(
          std::chrono::duration<double, std::micro>(c->t_launch - r->t_submit).count());
    if (s->inflight++ == 0) s->busy_since = c->t_launch;
    s->launches++;
    for (const auto &r : c->reqs) s->items += r->k;
    // the context's own thread issues the copies and kernels, so that
    // several contexts' launches are issued at once while this thread packs
    // the next
    c->ritem = std::move(ritem);
    c->rtiles = std::move(rtiles);
    c->pending = true;
    s->cv_issue.notify_all();
  }
}

// Issuing thread of context `ci`: runs the launches the scheduler packed
// into it (server lock not held while issuing).
static void issuer_loop(msrep_server *s, size_t ci) {
  cudaSetDevice(s->cfg.device);
  Context &c = s->ctx[ci];
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    s->cv_issue.wait(lk, [&] { return c.pending || s->stop_issuers; });
    if (!c.pending) return;  // stopping, nothing left to issue
    lk.unlock();
    const auto h0 = Clock::now();
    msrep_status st = launch_context(s, c, c.ritem, c.rtiles);
    const double host = std::chrono::duration<double, std::micro>(Clock::now() - h0).count();
    lk.lock();
    c.pending = false;
    s->host_us.push_back(host);
    if (st == MSREP_OK) c.in_flight = true;  // only now may its event be polled
    s->cv_flight.notify_all();
    if (st != MSREP_OK) {
      // fail the requests of this launch; the context stays usable
      cudaStreamSynchronize(c.stream);
      const std::string why = msrep_last_error();
      for (auto &r : c.reqs) {
        r->status = st;
        r->error = why;
        r->done = true;
        s->mats[r->matrix].refs--;
      }
      c.reqs.clear();
      c.busy = false;
      if (--s->inflight == 0)
        s->busy_s += std::chrono::duration<double>(Clock::now() - s->busy_since).count();
      s->cv_done.notify_all();
      s->cv_work.notify_all();
    }
  }
}

// Completion thread.  With nothing issued it sleeps on cv_flight; while
// any launch is in flight it polls the contexts' events back to back
// (yielding between sweeps): a timed sleep between polls would add the
// kernel's timer slack, tens of microseconds, to every request.
static void completion_loop(msrep_server *s) {
  cudaSetDevice(s->cfg.device);
  for (;;) {
    {
      std::unique_lock<std::mutex> lk(s->mu);
      bool any = false;
      s->cv_flight.wait(lk, [&] {
        bool flying = false;
        any = false;
        for (auto &c : s->ctx) {
          any |= c.busy;
          flying |= c.busy && c.in_flight;
        }
        return flying || (s->stop && s->queue.empty() && !any);
      });
      if (s->stop && s->queue.empty() && !any) return;
    }
    bool progressed = false;
    for (auto &c : s->ctx) {
      bool flying;
      {
        std::lock_guard<std::mutex> lk(s->mu);
        flying = c.busy && c.in_flight;
      }
      if (!flying) continue;
      const cudaError_t q = cudaEventQuery(c.done_ev);
      if (q == cudaErrorNotReady) continue;
      progressed = true;
      // results to the callers' buffers, outside the lock
      for (size_t i = 0; i < c.reqs.size(); ++i) {
        auto &r = c.reqs[i];
        int32_t m;
        {
          std::lock_guard<std::mutex> lk(s->mu);
          m = s->mats[r->matrix].m;
        }
        if (q == cudaSuccess && !r->y_pinned)
          std::memcpy(r->y, c.y_pin + c.y_off[i], sizeof(float) * size_t(m) * r->k);
      }
      float span_ms = 0.f, kern_ms = 0.f;
      const bool timed = q == cudaSuccess &&
                         cudaEventElapsedTime(&span_ms, c.begin_ev, c.done_ev) == cudaSuccess &&
                         cudaEventElapsedTime(&kern_ms, c.k0_ev, c.k1_ev) == cudaSuccess;
      const auto now = Clock::now();
      std::lock_guard<std::mutex> lk(s->mu);
      if (timed) {
        s->dev_us.push_back(1e3 * double(span_ms));
        s->kernel_us += 1e3 * double(kern_ms);
      }
      for (auto &r : c.reqs) {
        r->status = q == cudaSuccess ? MSREP_OK : MSREP_ERR_CUDA;
        if (q != cudaSuccess) r->error = cudaGetErrorString(q);
        r->done = true;
        s->mats[r->matrix].refs--;
        s->lat_us.push_back(std::chrono::duration<double, std::micro>(now - r->t_submit).count());
        s->completed++;
      }
      s->work_bytes += c.bytes;
      c.reqs.clear();
      c.busy = false;
      c.in_flight = false;
      if (--s->inflight == 0)
        s->busy_s += std::chrono::duration<double>(now - s->busy_since).count();
      s->cv_done.notify_all();
      s->cv_work.notify_all();
    }
    if (!progressed) std::this_thread::yield();
  }
}

}  // namespace msrep

using namespace msrep;

extern "C" {

msrep_status msrep_serve_config_default(msrep_serve_config *c) {
  if (!c) return fail(MSREP_ERR_INVALID_ARG, "cfg is NULL");
  c->budget_bytes = int64_t(60) << 30;
  c->arena_bytes = int64_t(64) << 20;
  c->contexts = 3;
  c->max_items = 256;
  c->max_k = 8;
  c->tile = 0;
  c->max_tiles = int64_t(1) << 20;
  c->device = 0;
  return ok();
}

msrep_status msrep_serve_create(const msrep_serve_config *cfg, msrep_server **out) {
  if (!cfg || !out) return fail(MSREP_ERR_INVALID_ARG, "cfg or out is NULL");
  if (cfg->contexts < 1 || cfg->max_items < 1 || cfg->max_k < 1 || cfg->max_k > kBatchWidth ||
      cfg->arena_bytes < 4096 || cfg->max_tiles < 1 || !tile_supported(effective_tile(cfg->tile)))
    return fail(MSREP_ERR_INVALID_ARG, "bad serve config");
  // x, y arenas; interleaved-x arena (8 values per column: up to four times
  // the x of a request with two vectors); directories; partials of both
  // kernels
  const int64_t per_ctx = 2 * align256(cfg->arena_bytes) + 4 * align256(cfg->arena_bytes) +
                          int64_t(dir_size(cfg->max_items)) +
                          2 * int64_t(align256(sizeof(double) * cfg->max_tiles)) +
                          2 * int64_t(align256(sizeof(double) * cfg->max_tiles * kBatchWidth));
  if (per_ctx * cfg->contexts > cfg->budget_bytes)
    return fail(MSREP_ERR_BUDGET, "the launch contexts alone exceed the budget");
  MSREP_CUDA_TRY(cudaSetDevice(cfg->device));
  auto s = std::make_unique<msrep_server>();
  s->cfg = *cfg;
  s->ctx.resize(cfg->contexts);
  for (auto &c : s->ctx) {
    c.arena_floats = cfg->arena_bytes / int64_t(sizeof(float));
    c.max_tiles = cfg->max_tiles;
    c.dir_bytes = dir_size(cfg->max_items);
    c.xt_floats = 4 * cfg->arena_bytes / int64_t(sizeof(float));
    bool okc = cudaStreamCreateWithFlags(&c.stream, cudaStreamNonBlocking) == cudaSuccess &&
               cudaEventCreate(&c.done_ev) == cudaSuccess &&
               cudaEventCreate(&c.begin_ev) == cudaSuccess &&
               cudaEventCreate(&c.k0_ev) == cudaSuccess &&
               cudaEventCreate(&c.k1_ev) == cudaSuccess &&
               cudaMalloc(&c.x_dev, cfg->arena_bytes) == cudaSuccess &&
               cudaMalloc(&c.y_dev, cfg->arena_bytes) == cudaSuccess &&
               cudaMalloc(&c.dir_dev, c.dir_bytes) == cudaSuccess &&
               cudaMalloc(&c.head, sizeof(double) * cfg->max_tiles) == cudaSuccess &&
               cudaMalloc(&c.tail, sizeof(double) * cfg->max_tiles) == cudaSuccess &&
               cudaMallocHost(&c.x_pin, cfg->arena_bytes) == cudaSuccess &&
               cudaMallocHost(&c.y_pin, cfg->arena_bytes) == cudaSuccess &&
               cudaMallocHost(&c.dir_pin, c.dir_bytes) == cudaSuccess &&
               cudaMalloc(&c.xt_dev, sizeof(float) * c.xt_floats) == cudaSuccess &&
               cudaMalloc(&c.head_k, sizeof(double) * cfg->max_tiles * kBatchWidth) == cudaSuccess &&
               cudaMalloc(&c.tail_k, sizeof(double) * cfg->max_tiles * kBatchWidth) == cudaSuccess &&
               true;
    if (!okc) {
      for (auto &cc : s->ctx) free_context(cc);
      cudaGetLastError();
      return fail(MSREP_ERR_OOM, "cannot allocate the launch contexts");
    }
  }
  s->resident = per_ctx * cfg->contexts;
  msrep_server *raw = s.release();
  raw->scheduler = std::thread(scheduler_loop, raw);
  for (size_t ci = 0; ci < raw->ctx.size(); ++ci) raw->issuers.emplace_back(issuer_loop, raw, ci);
  raw->completer = std::thread(completion_loop, raw);
  *out = raw;
  return ok();
}

msrep_status msrep_serve_register(msrep_server *s, const msrep_matrix *A, int64_t *matrix_id) {
  if (!s || !A || !matrix_id) return fail(MSREP_ERR_INVALID_ARG, "NULL argument");
  if (A->fmt != MSREP_CSR || !A->ptr || (A->nnz > 0 && (!A->idx || !A->val)) || A->m < 0 ||
      A->n < 0 || A->nnz < 0 || A->nnz > INT32_MAX || A->val_dtype < MSREP_F64 ||
      A->val_dtype > MSREP_BF16)
    return fail(MSREP_ERR_INVALID_ARG, "register needs a CSR matrix with host arrays");
  MSREP_CUDA_TRY(cudaSetDevice(s->cfg.device));
  const int32_t tile = effective_tile(s->cfg.tile);
  const int32_t np = static_cast<int32_t>(std::max<int64_t>(1, ceil_div(A->nnz, int64_t(1) << 20)));
  const PlanLayout PL = plan_layout(A->m, A->nnz, np, tile);
  size_t o = 0;
  const size_t o_ptr = o;  o = align256(o + sizeof(int32_t) * (size_t(A->m) + 1));
  const size_t o_col = o;  o = align256(o + sizeof(int32_t) * size_t(A->nnz));
  const size_t o_val = o;  o = align256(o + sizeof(float) * size_t(A->nnz));
  const size_t o_meta = o; o = align256(o + 4 * sizeof(int32_t) * size_t(np));
  const size_t o_flag = o; o = align256(o + size_t(np));
  const size_t o_plan = o; o = align256(o + PL.bytes);
  const size_t bytes = o;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) return fail(MSREP_ERR_SHUTDOWN, "server is stopping");
    if (s->resident + int64_t(bytes) > s->cfg.budget_bytes) {
      s->rejected++;
      return fail(MSREP_ERR_BUDGET, "matrix needs %zu bytes, %lld of %lld in use", bytes,
                  (long long)s->resident, (long long)s->cfg.budget_bytes);
    }
    s->resident += int64_t(bytes);  // reserve
  }
  void *mem = nullptr;
  auto unreserve = [&](msrep_status st) {
    std::lock_guard<std::mutex> lk(s->mu);
    s->resident -= int64_t(bytes);
    if (mem) cudaFree(mem);
    return st;
  };
  if (cudaMalloc(&mem, bytes) != cudaSuccess) {
    cudaGetLastError();
    return unreserve(fail(MSREP_ERR_OOM, "device allocation of %zu bytes failed", bytes));
  }
  char *b = static_cast<char *>(mem);
  // values to FP32 on the host
  std::vector<float> vf(size_t(A->nnz));
  for (int64_t k = 0; k < A->nnz; ++k) {
    if (A->val_dtype == MSREP_F64)
      vf[k] = static_cast<float>(static_cast<const double *>(A->val)[k]);
    else if (A->val_dtype == MSREP_F32)
      vf[k] = static_cast<const float *>(A->val)[k];
    else {
      uint32_t w = uint32_t(static_cast<const uint16_t *>(A->val)[k]) << 16;
      std::memcpy(&vf[k], &w, 4);
    }
  }
  cudaStream_t st = nullptr;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess)
    return unreserve(fail(MSREP_ERR_CUDA, "stream creation failed"));
  bool good = cudaMemcpyAsync(b + o_ptr, A->ptr, sizeof(int32_t) * (size_t(A->m) + 1),
                              cudaMemcpyHostToDevice, st) == cudaSuccess &&
              (A->nnz == 0 ||
               (cudaMemcpyAsync(b + o_col, A->idx, sizeof(int32_t) * size_t(A->nnz),
                                cudaMemcpyHostToDevice, st) == cudaSuccess &&
                cudaMemcpyAsync(b + o_val, vf.data(), sizeof(float) * size_t(A->nnz),
                                cudaMemcpyHostToDevice, st) == cudaSuccess));
  msrep_matrix D = *A;
  D.val_dtype = MSREP_F32;
  D.ptr = reinterpret_cast<const int32_t *>(b + o_ptr);
  D.idx = reinterpret_cast<const int32_t *>(b + o_col);
  D.val = b + o_val;
  msrep_partition p{};
  p.np = np;
  p.tile = tile;
  int32_t *meta = reinterpret_cast<int32_t *>(b + o_meta);
  p.start_idx = meta;
  p.end_idx = meta + np;
  p.start_major = meta + 2 * np;
  p.end_major = meta + 3 * np;
  p.start_flag = reinterpret_cast<uint8_t *>(b + o_flag);
  p.plan = b + o_plan;
  p.plan_bytes = static_cast<int64_t>(PL.bytes);
  int32_t ntiles = 0;
  if (good) good = msrep_partition_csr(&D, &p, 0, st) == MSREP_OK;
  if (good)
    good = cudaMemcpyAsync(&ntiles, b + o_plan + PL.off_toff + sizeof(int32_t) * np,
                           sizeof(int32_t), cudaMemcpyDeviceToHost, st) == cudaSuccess &&
           cudaStreamSynchronize(st) == cudaSuccess;
  cudaStreamDestroy(st);
  if (!good) {
    cudaGetLastError();
    return unreserve(fail(MSREP_ERR_CUDA, "upload or partition failed"));
  }
  Resident R;
  R.m = A->m;
  R.n = A->n;
  R.nnz = A->nnz;
  R.np = np;
  R.tile = tile;
  R.tiles = ntiles;
  R.mem = mem;
  R.bytes = bytes;
  R.item = BatchItem{D.ptr, D.idx, D.val, reinterpret_cast<const int32_t *>(b + o_plan + PL.off_row),
                     reinterpret_cast<const int32_t *>(b + o_plan + PL.off_k), A->m, A->n, A->nnz,
                     1, 0};
  std::lock_guard<std::mutex> lk(s->mu);
  R.id = s->next_matrix++;
  *matrix_id = R.id;
  s->mats[R.id] = R;
  return ok();
}

msrep_status msrep_serve_unregister(msrep_server *s, int64_t id) {
  if (!s) return fail(MSREP_ERR_INVALID_ARG, "server is NULL");
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->mats.find(id);
  if (it == s->mats.end() || it->second.dying) return fail(MSREP_ERR_NOT_FOUND, "unknown matrix %lld", (long long)id);
  it->second.dying = true;
  s->cv_done.wait(lk, [&] { return it->second.refs == 0; });
  cudaFree(it->second.mem);
  s->resident -= int64_t(it->second.bytes);
  s->mats.erase(it);
  return ok();
}

msrep_status msrep_serve_submit(msrep_server *s, int64_t id, int32_t k, const float *x,
                                float *y, uint64_t *req_id) {
  if (!s || !x || !y || !req_id) return fail(MSREP_ERR_INVALID_ARG, "NULL argument");
  if (k < 1 || k > s->cfg.max_k) return fail(MSREP_ERR_INVALID_ARG, "k must be 1..%d", s->cfg.max_k);
  auto r = std::make_shared<Request>();
  r->matrix = id;
  r->k = k;
  r->x = x;
  r->y = y;
  r->t_submit = Clock::now();
  {
    // page-locked caller buffers are copied by DMA without a staging copy,
    // and read / written by the launch's kernels directly when they are
    // mapped at the same address (unified addressing), the only mapping
    // used here
    auto mapped = [](const void *p, bool &pinned) -> const void * {
      cudaPointerAttributes at;
      pinned = cudaPointerGetAttributes(&at, p) == cudaSuccess && at.type == cudaMemoryTypeHost;
      if (!pinned || !at.devicePointer || !at.hostPointer) return nullptr;
      const void *d = static_cast<const char *>(at.devicePointer) +
                      (static_cast<const char *>(p) - static_cast<const char *>(at.hostPointer));
      return d == p ? p : nullptr;
    };
    r->x_map = static_cast<const float *>(mapped(x, r->x_pinned));
    r->y_map = static_cast<float *>(const_cast<void *>(mapped(y, r->y_pinned)));
    cudaGetLastError();
  }
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->stop) return fail(MSREP_ERR_SHUTDOWN, "server is stopping");
  auto it = s->mats.find(id);
  if (it == s->mats.end() || it->second.dying)
    return fail(MSREP_ERR_NOT_FOUND, "unknown matrix %lld", (long long)id);
  const int64_t nx = int64_t(it->second.n) * k, ny = int64_t(it->second.m) * k;
  const int64_t cap = s->cfg.arena_bytes / int64_t(sizeof(float));
  if (nx > cap || ny > cap || it->second.tiles * k > s->cfg.max_tiles)
    return fail(MSREP_ERR_INVALID_ARG, "request does not fit one launch context");
  it->second.refs++;
  r->id = s->next_req++;
  *req_id = r->id;
  s->reqs[r->id] = r;
  s->queue.push_back(r);
  s->submitted++;
  s->cv_work.notify_one();
  return ok();
}

msrep_status msrep_serve_wait(msrep_server *s, uint64_t req_id, int64_t timeout_us) {
  if (!s) return fail(MSREP_ERR_INVALID_ARG, "server is NULL");
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(req_id);
  if (it == s->reqs.end()) return fail(MSREP_ERR_NOT_FOUND, "unknown request %llu", (unsigned long long)req_id);
  auto r = it->second;
  if (timeout_us < 0) {
    s->cv_done.wait(lk, [&] { return r->done; });
  } else if (!s->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), [&] { return r->done; })) {
    return fail(MSREP_ERR_TIMEOUT, "request %llu not finished", (unsigned long long)req_id);
  }
  s->reqs.erase(req_id);
  if (r->status != MSREP_OK)
    return fail(r->status, "request %llu failed: %s", (unsigned long long)req_id, r->error.c_str());
  return ok();
}

msrep_status msrep_serve_replay(msrep_server *s, int64_t count, const double *t_us,
                                const int64_t *matrix_id, const int32_t *k,
                                const float *const *x, float *const *y, const int64_t *reuse,
                                double reset_after_us, int64_t *late, double *max_lag_us) {
  if (!s || count < 0 || (count > 0 && (!t_us || !matrix_id || !k || !x || !y || !reuse)) ||
      !late || !max_lag_us)
    return fail(MSREP_ERR_INVALID_ARG, "NULL argument or negative count");
  for (int64_t i = 0; i < count; ++i)
    if (reuse[i] >= i || (i > 0 && t_us[i] < t_us[i - 1]))
      return fail(MSREP_ERR_INVALID_ARG,
                  "arrival times must not decrease and reuse[i] must be < i (request %lld)",
                  (long long)i);
  std::vector<uint64_t> ids(static_cast<size_t>(count), 0);
  std::vector<char> collected(static_cast<size_t>(count), 0);
  *late = 0;
  *max_lag_us = 0.0;
  bool reset_done = reset_after_us < 0;
  msrep_status status = MSREP_OK;
  const auto t0 = Clock::now();
  auto since = [&] { return std::chrono::duration<double, std::micro>(Clock::now() - t0).count(); };
  for (int64_t i = 0; i < count && status == MSREP_OK; ++i) {
    // the request that last used this request's buffers must be done
    const int64_t d = reuse[i];
    if (d >= 0 && !collected[d]) {
      status = msrep_serve_wait(s, ids[d], -1);
      collected[d] = 1;
      if (status != MSREP_OK) break;
    }
    while (since() < t_us[i]) {
    }
    if (!reset_done && since() >= reset_after_us) {
      msrep_serve_counters tmp;
      msrep_serve_stats(s, &tmp, 1);
      reset_done = true;
    }
    const double lag = since() - t_us[i];
    if (lag > 100.0) ++*late;
    *max_lag_us = std::max(*max_lag_us, lag);
    status = msrep_serve_submit(s, matrix_id[i], k[i], x[i], y[i], &ids[i]);
  }
  for (int64_t i = 0; i < count; ++i)
    if (ids[i] && !collected[i]) {
      const msrep_status w = msrep_serve_wait(s, ids[i], -1);
      if (status == MSREP_OK) status = w;
    }
  if (status != MSREP_OK) return status;
  return ok();
}

msrep_status msrep_serve_stats(msrep_server *s, msrep_serve_counters *o, int32_t reset) {
  if (!s || !o) return fail(MSREP_ERR_INVALID_ARG, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  std::memset(o, 0, sizeof *o);
  o->submitted = s->submitted;
  o->completed = s->completed;
  o->rejected = s->rejected;
  o->launches = s->launches;
  // percentile p of a sample (nearest rank), 0 when empty
  auto pct = [](std::vector<double> v, double p) {
    if (v.empty()) return 0.0;
    std::sort(v.begin(), v.end());
    return v[std::min(v.size() - 1, size_t(p * (v.size() - 1) + 0.5))];
  };
  const std::vector<double> &l = s->lat_us;
  if (!l.empty()) {
    o->p50_us = pct(l, 0.50);
    o->p99_us = pct(l, 0.99);
    double sum = 0, mx = 0;
    for (double v : l) {
      sum += v;
      mx = std::max(mx, v);
    }
    o->mean_us = sum / l.size();
    o->max_us = mx;
  }
  o->wait_p50_us = pct(s->wait_us, 0.50);
  o->wait_p99_us = pct(s->wait_us, 0.99);
  o->device_p50_us = pct(s->dev_us, 0.50);
  o->device_p99_us = pct(s->dev_us, 0.99);
  o->kernel_mean_us = s->dev_us.empty() ? 0.0 : s->kernel_us / double(s->dev_us.size());
  o->host_launch_p50_us = pct(s->host_us, 0.50);
  o->host_launch_p99_us = pct(s->host_us, 0.99);
  double busy = s->busy_s;
  if (s->inflight > 0) busy += std::chrono::duration<double>(Clock::now() - s->busy_since).count();
  o->busy_s = busy;
  o->gbs = busy > 0 ? s->work_bytes / busy / 1e9 : 0.0;
  o->mean_items = s->launches ? double(s->items) / double(s->launches) : 0.0;
  o->resident_bytes = s->resident;
  if (reset) {
    s->lat_us.clear();
    s->wait_us.clear();
    s->dev_us.clear();
    s->host_us.clear();
    s->kernel_us = 0;
    s->submitted = s->completed = s->rejected = s->launches = s->items = 0;
    s->work_bytes = 0;
    s->busy_s = 0;
    if (s->inflight > 0) s->busy_since = Clock::now();
  }
  return ok();
}

msrep_status msrep_serve_destroy(msrep_server *s) {
  if (!s) return fail(MSREP_ERR_INVALID_ARG, "server is NULL");
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->cv_work.notify_all();
    s->cv_flight.notify_all();
  }
  if (s->scheduler.joinable()) s->scheduler.join();
  {
    // every packed launch is issued before the issuing threads stop
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop_issuers = true;
    s->cv_issue.notify_all();
    s->cv_flight.notify_all();
  }
  for (auto &t : s->issuers)
    if (t.joinable()) t.join();
  if (s->completer.joinable()) s->completer.join();
  for (auto &c : s->ctx) free_context(c);
  for (auto &kv : s->mats) cudaFree(kv.second.mem);
  delete s;
  return ok();
}

}  // extern "C"
