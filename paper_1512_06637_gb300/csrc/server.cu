// server.cu -- continuous-batching service for navigation requests.
//
// The scheduler of the paper (Project goals, item 1) keeps feeding baskets of
// particles to the geometry.  Here a request is a basket of tracks (world points
// and directions) that needs locate + one navigation step.  A worker thread owns
// the device side:
//   * admission: FIFO requests are admitted while a slot is free and the device
//     arena has room for the request (72 bytes per track); a request that can
//     never fit is refused at submit time;
//   * batching: everything admitted in one pass of the worker forms a group that
//     shares one launch of each kernel (unpack -> locate -> navigation step ->
//     pack), so requests that arrive while others are on the GPU join the next
//     group;
//   * overlap: groups go round-robin to several streams, so the copies of one
//     group overlap the kernels of another;
//   * completion: an event per group; the worker marks its requests done when the
//     host sees the event, frees the arena in issue order, and records the
//     latency from submit to completion.
// Request buffers are host memory (pinned for speed): input 6 n doubles
// (x, y, z, dx, dy, dz blocks of n), output 2 n doubles + 2 n int32 (step,
// safety, next, node blocks).  No device wait spins: the worker polls events
// from the host and sleeps briefly when idle.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>
#include "gv_internal.h"

namespace gv {

constexpr int64_t kBytesPerTrack = 6 * 8 + 4 + 2 * 8 + 4;  // in + node + step, safety + next
constexpr int kMaxStreams = 8;

struct Seg {          // one request inside a group
  long long stage;    // offset of its packed input in the staging area (doubles)
  long long n;
  long long gofs;     // first track in the group's SoA arrays
};

// staging (per-request packed input) -> group SoA arrays
__global__ void k_unpack(const double* __restrict__ stage, const Seg* __restrict__ segs, int nseg,
                         double* __restrict__ soa, long long gn) {
  for (int s = blockIdx.y; s < nseg; s += gridDim.y) {
    const Seg g = segs[s];
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < g.n; j += (long long)gridDim.x * blockDim.x)
      for (int c = 0; c < 6; c++) soa[c * gn + g.gofs + j] = stage[g.stage + c * g.n + j];
  }
}
// group results -> per-request packed output (step, safety as doubles; next, node as int32)
__global__ void k_pack(const double* __restrict__ step, const double* __restrict__ saf, const int32_t* __restrict__ next,
                       const int32_t* __restrict__ node, const Seg* __restrict__ segs, int nseg,
                       unsigned char* __restrict__ outbuf) {
  for (int s = blockIdx.y; s < nseg; s += gridDim.y) {
    const Seg g = segs[s];
    // the packed output of a request sits at 24 * (its staging offset / 6) bytes
    double* o = reinterpret_cast<double*>(outbuf + (size_t)(g.stage / 6) * 24);
    int32_t* oi = reinterpret_cast<int32_t*>(o + 2 * g.n);
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < g.n; j += (long long)gridDim.x * blockDim.x) {
      o[j] = step[g.gofs + j];
      o[g.n + j] = saf[g.gofs + j];
      oi[j] = next[g.gofs + j];
      oi[g.n + j] = node[g.gofs + j];
    }
  }
}

}  // namespace gv

using namespace gv;
using Clock = std::chrono::steady_clock;

struct Request {
  int64_t ticket;
  int64_t n;
  const double* in;
  void* out;
  Clock::time_point t_submit;
  double latency_ms = -1;
  bool done = false;
  int64_t group = -1;
};

struct Group {
  int64_t id;
  int stream;
  int64_t arena_off, arena_len;   // bytes of the ring used by this group
  cudaEvent_t done;
  std::vector<int64_t> tickets;
  bool finished = false;
};

struct gv_server {
  const gv_geom* geom;
  gv_server_config cfg;
  int device;
  // device memory
  unsigned char* arena = nullptr;   // ring of group regions
  int64_t arena_bytes = 0;
  int64_t ring_head = 0, ring_tail = 0, ring_used = 0;  // bytes; allocations at tail, frees at head
  Seg* d_segs = nullptr;            // per stream, max_slots entries
  Seg* h_segs = nullptr;            // pinned, per stream
  cudaStream_t streams[kMaxStreams] = {};
  cudaEvent_t seg_ready[kMaxStreams] = {};  // the stream's segment table has been copied
  gv_workspace* ws[kMaxStreams] = {};
  int next_stream = 0;
  // host state
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<int64_t> queue;                 // submitted, not yet admitted
  std::unordered_map<int64_t, Request> reqs;  // live requests
  std::deque<Group> inflight;                 // issue order
  int64_t next_ticket = 1, next_group = 1;
  int slots_used = 0;
  std::vector<double> lat_ms;                 // completed latencies
  int64_t completed = 0, tracks_done = 0, launches = 0;
  std::atomic<bool> stop{false};
  gv_status worker_status = GV_OK;
  std::thread worker;
};

static int64_t align256(int64_t v) { return (v + 255) & ~(int64_t)255; }

// bytes of arena a group of total n tracks needs: packed staging (48 n) + SoA in (48 n)
// + node (4 n) + step, safety (16 n) + next (4 n) + packed out (24 n)
static int64_t group_bytes(int64_t n) {
  return align256(48 * n) + align256(48 * n) + align256(4 * n) + align256(16 * n) + align256(4 * n) + align256(24 * n) + 256;
}

// Ring allocation of len bytes; returns offset or -1.
static int64_t ring_alloc(gv_server* s, int64_t len) {
  if (len > s->arena_bytes || s->ring_used + len > s->arena_bytes) return -1;
  if (s->ring_used == 0) { s->ring_head = s->ring_tail = 0; }
  if (s->ring_tail >= s->ring_head && s->ring_used > 0) {
    if (s->arena_bytes - s->ring_tail >= len) { int64_t o = s->ring_tail; s->ring_tail += len; s->ring_used += len; return o; }
    if (s->ring_head >= len) { s->ring_used += (s->arena_bytes - s->ring_tail) + len; s->ring_tail = len; return 0; }
    return -1;
  }
  if (s->ring_used == 0) {
    s->ring_tail = len; s->ring_used = len; return 0;
  }
  // wrapped: free space is [tail, head)
  if (s->ring_head - s->ring_tail >= len) { int64_t o = s->ring_tail; s->ring_tail += len; s->ring_used += len; return o; }
  return -1;
}

static void ring_free_head(gv_server* s, const Group& g) {
  // groups are freed in issue order; account the bytes from the group start (and a skipped end gap)
  int64_t len = g.arena_len;
  if (g.arena_off != s->ring_head) len += s->arena_bytes - s->ring_head;  // the wrap gap
  s->ring_used -= len;
  s->ring_head = g.arena_off + g.arena_len;
  if (s->ring_used <= 0) { s->ring_used = 0; s->ring_head = s->ring_tail = 0; }
}

static gv_status issue_group(gv_server* s, std::vector<int64_t>& tickets, int64_t total, int64_t off) {
  const gv::Range range("gv_server group");
  const int si = s->next_stream;
  s->next_stream = (s->next_stream + 1) % s->cfg.streams;
  cudaStream_t st = s->streams[si];
  unsigned char* base = s->arena + off;
  double* stage = reinterpret_cast<double*>(base);
  unsigned char* p = base + align256(48 * total);
  double* soa = reinterpret_cast<double*>(p); p += align256(48 * total);
  int32_t* node = reinterpret_cast<int32_t*>(p); p += align256(4 * total);
  double* step = reinterpret_cast<double*>(p); p += align256(8 * total);
  double* saf = step + total; p += align256(16 * total) - align256(8 * total);
  int32_t* next = reinterpret_cast<int32_t*>(p); p += align256(4 * total);
  unsigned char* packed = p;
  Seg* hs = s->h_segs + (size_t)si * s->cfg.max_slots;
  Seg* ds = s->d_segs + (size_t)si * s->cfg.max_slots;
  // the previous group on this stream may still be copying hs: wait for that copy only
  cudaEventSynchronize(s->seg_ready[si]);
  long long stage_off = 0, gofs = 0;
  int nseg = 0;
  cudaError_t e = cudaSuccess;
  for (int64_t t : tickets) {
    Request& r = s->reqs[t];
    hs[nseg] = Seg{stage_off, r.n, gofs};
    if (r.n > 0) e = cudaMemcpyAsync(stage + stage_off, r.in, 48 * r.n, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_error(e, "server: request copy in");
    stage_off += 6 * r.n;
    gofs += r.n;
    nseg++;
  }
  e = cudaMemcpyAsync(ds, hs, sizeof(Seg) * nseg, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaEventRecord(s->seg_ready[si], st);
  if (e != cudaSuccess) return cuda_error(e, "server: segment table");
  const int sms = sm_count();
  if (total > 0) {
    dim3 grid((unsigned)std::min<int64_t>((total / std::max(nseg, 1) + 255) / 256 + 1, 64), (unsigned)std::min(nseg, 1024));
    k_unpack<<<grid, 256, 0, st>>>(stage, ds, nseg, soa, total);
    gv_tracks tr{soa, soa + total, soa + 2 * total, soa + 3 * total, soa + 4 * total, soa + 5 * total, total};
    gv_status gs = gv_nav_locate(s->geom, &tr, node, st);
    if (gs != GV_OK) return gs;
    gs = gv_nav_step(s->geom, &tr, node, (gv_precision)s->cfg.precision, step, saf, next, s->ws[si], st);
    if (gs != GV_OK) return gs;
    k_pack<<<grid, 256, 0, st>>>(step, saf, next, node, ds, nseg, packed);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "server: kernels");
    (void)sms;
  }
  for (int k = 0; k < nseg; k++) {
    Request& r = s->reqs[tickets[k]];
    if (r.n > 0) e = cudaMemcpyAsync(r.out, packed + (size_t)(hs[k].stage / 6) * 24, 24 * r.n, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return cuda_error(e, "server: result copy out");
  }
  Group g;
  g.id = s->next_group++;
  g.stream = si;
  g.arena_off = off;
  g.arena_len = group_bytes(total);
  g.tickets = tickets;
  e = cudaEventCreateWithFlags(&g.done, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(g.done, st);
  if (e != cudaSuccess) return cuda_error(e, "server: completion event");
  for (int64_t t : tickets) s->reqs[t].group = g.id;
  s->inflight.push_back(g);
  s->launches++;
  return GV_OK;
}

static void worker_loop(gv_server* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  while (true) {
    // retire finished groups
    bool progressed = false;
    for (Group& g : s->inflight) {
      if (g.finished) continue;
      const cudaError_t q = cudaEventQuery(g.done);
      if (q == cudaSuccess) {
        g.finished = true;
        const auto now = Clock::now();
        for (int64_t t : g.tickets) {
          Request& r = s->reqs[t];
          r.done = true;
          r.latency_ms = std::chrono::duration<double, std::milli>(now - r.t_submit).count();
          s->lat_ms.push_back(r.latency_ms);
          s->completed++;
          s->tracks_done += r.n;
          s->slots_used--;
        }
        progressed = true;
      } else if (q != cudaErrorNotReady) {
        s->worker_status = cuda_error(q, "server: group failed");
        g.finished = true;
        for (int64_t t : g.tickets) { s->reqs[t].done = true; s->slots_used--; }
        progressed = true;
      }
    }
    while (!s->inflight.empty() && s->inflight.front().finished) {
      ring_free_head(s, s->inflight.front());
      cudaEventDestroy(s->inflight.front().done);
      s->inflight.pop_front();
    }
    if (progressed) s->cv_done.notify_all();
    // admit: everything that fits now forms one group
    std::vector<int64_t> admit;
    int64_t total = 0;
    while (!s->queue.empty() && s->slots_used + (int)admit.size() < s->cfg.max_slots) {
      const int64_t t = s->queue.front();
      const int64_t n = s->reqs[t].n;
      if (group_bytes(total + n) > s->arena_bytes) break;
      admit.push_back(t);
      total += n;
      s->queue.pop_front();
    }
    if (!admit.empty()) {
      int64_t off = ring_alloc(s, group_bytes(total));
      if (off < 0) {  // not enough contiguous room yet: put them back, wait for completions
        for (auto it = admit.rbegin(); it != admit.rend(); ++it) s->queue.push_front(*it);
      } else {
        s->slots_used += (int)admit.size();
        gv_status st = issue_group(s, admit, total, off);
        if (st != GV_OK) s->worker_status = st;
        continue;
      }
    }
    if (s->stop && s->queue.empty() && s->inflight.empty()) break;
    if (s->inflight.empty() && s->queue.empty()) s->cv_work.wait_for(lk, std::chrono::milliseconds(5));
    else {
      lk.unlock();
      std::this_thread::sleep_for(std::chrono::microseconds(20));
      lk.lock();
    }
  }
}

extern "C" {

gv_status gv_server_create(const gv_geom* g, const gv_server_config* cfg, gv_server** out) {
  if (!g || !cfg || !out) return set_error(GV_ERR_INVALID_ARG, "server: NULL argument");
  if (cfg->arena_bytes < (1 << 16)) return set_error(GV_ERR_INVALID_ARG, "server: arena below 64 KiB");
  if (cfg->max_slots < 1 || cfg->max_slots > 65536) return set_error(GV_ERR_INVALID_ARG, "server: max_slots in 1..65536");
  if (cfg->streams < 1 || cfg->streams > kMaxStreams) return set_error(GV_ERR_INVALID_ARG, "server: streams in 1..8");
  if (cfg->precision != GV_FP64 && cfg->precision != GV_FP32_REFINE) return set_error(GV_ERR_INVALID_ARG, "server: precision");
  gv_server* s = new (std::nothrow) gv_server;
  if (!s) return set_error(GV_ERR_OUT_OF_MEMORY, "host allocation failed");
  s->geom = g;
  s->cfg = *cfg;
  s->arena_bytes = cfg->arena_bytes;
  cudaError_t e = cudaGetDevice(&s->device);
  if (e == cudaSuccess) e = cudaMalloc(&s->arena, s->arena_bytes);
  if (e == cudaSuccess) e = cudaMalloc(&s->d_segs, sizeof(Seg) * cfg->max_slots * cfg->streams);
  if (e == cudaSuccess) e = cudaMallocHost(&s->h_segs, sizeof(Seg) * cfg->max_slots * cfg->streams);
  for (int i = 0; i < cfg->streams && e == cudaSuccess; i++) {
    e = cudaStreamCreateWithFlags(&s->streams[i], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->seg_ready[i], cudaEventDisableTiming);
  }
  gv_status st = GV_OK;
  if (e != cudaSuccess) st = e == cudaErrorMemoryAllocation ? set_error(GV_ERR_OUT_OF_MEMORY, "server: allocation failed")
                                                           : cuda_error(e, "server create");
  const int64_t max_tracks = s->arena_bytes / kBytesPerTrack + 1;
  for (int i = 0; i < cfg->streams && st == GV_OK; i++) st = gv_workspace_create(max_tracks, &s->ws[i]);
  if (st != GV_OK) {
    gv_server_destroy(s);
    return st;
  }
  s->worker = std::thread(worker_loop, s);
  *out = s;
  return GV_OK;
}

gv_status gv_server_submit(gv_server* s, int64_t n, const double* host_in, void* host_out, int64_t* ticket) {
  const gv::Range range("gv_server_submit");
  if (!s || !ticket || n < 0 || (n > 0 && (!host_in || !host_out)))
    return set_error(GV_ERR_INVALID_ARG, "server submit: bad arguments");
  if (group_bytes(n) > s->arena_bytes)
    return set_error(GV_ERR_OUT_OF_MEMORY, "server submit: request larger than the device arena");
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->worker_status != GV_OK) return s->worker_status;
  Request r;
  r.ticket = s->next_ticket++;
  r.n = n;
  r.in = host_in;
  r.out = host_out;
  r.t_submit = Clock::now();
  s->reqs.emplace(r.ticket, r);
  s->queue.push_back(r.ticket);
  *ticket = r.ticket;
  s->cv_work.notify_one();
  return GV_OK;
}

gv_status gv_server_poll(gv_server* s, int64_t ticket, int32_t* done) {
  if (!s || !done) return set_error(GV_ERR_INVALID_ARG, "server poll: NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return set_error(GV_ERR_INVALID_ARG, "server poll: unknown ticket");
  *done = it->second.done ? 1 : 0;
  return s->worker_status;
}

gv_status gv_server_wait(gv_server* s, int64_t ticket, double timeout_s, double* latency_ms) {
  if (!s) return set_error(GV_ERR_INVALID_ARG, "server wait: NULL server");
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return set_error(GV_ERR_INVALID_ARG, "server wait: unknown ticket");
  const auto deadline = Clock::now() + std::chrono::duration<double>(timeout_s > 0 ? timeout_s : 0);
  while (!s->reqs[ticket].done) {
    if (s->worker_status != GV_OK) return s->worker_status;
    if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && !s->reqs[ticket].done)
      return set_error(GV_ERR_TIMEOUT, "server wait: timed out");
  }
  if (latency_ms) *latency_ms = s->reqs[ticket].latency_ms;
  s->reqs.erase(ticket);  // a waited ticket is released
  return s->worker_status;
}

gv_status gv_server_get_stats(gv_server* s, gv_server_stats* out) {
  if (!s || !out) return set_error(GV_ERR_INVALID_ARG, "server stats: NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  out->completed = s->completed;
  out->tracks = s->tracks_done;
  out->launches = s->launches;
  out->queued = (int64_t)s->queue.size();
  std::vector<double> v = s->lat_ms;
  std::sort(v.begin(), v.end());
  auto q = [&](double f) { return v.empty() ? 0.0 : v[std::min(v.size() - 1, (size_t)(f * (v.size() - 1) + 0.5))]; };
  out->p50_ms = q(0.5);
  out->p99_ms = q(0.99);
  out->max_ms = v.empty() ? 0.0 : v.back();
  double sum = 0;
  for (double x : v) sum += x;
  out->mean_ms = v.empty() ? 0.0 : sum / v.size();
  return GV_OK;
}

gv_status gv_server_reset_stats(gv_server* s) {
  if (!s) return set_error(GV_ERR_INVALID_ARG, "server: NULL");
  std::lock_guard<std::mutex> lk(s->mu);
  s->lat_ms.clear();
  s->completed = s->tracks_done = s->launches = 0;
  return GV_OK;
}

void gv_server_destroy(gv_server* s) {
  if (!s) return;
  if (s->worker.joinable()) {
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->stop = true;
    }
    s->cv_work.notify_all();
    s->worker.join();
  }
  for (Group& g : s->inflight) { cudaEventSynchronize(g.done); cudaEventDestroy(g.done); }
  for (int i = 0; i < kMaxStreams; i++) {
    if (s->seg_ready[i]) cudaEventDestroy(s->seg_ready[i]);
    if (s->streams[i]) cudaStreamDestroy(s->streams[i]);
    if (s->ws[i]) gv_workspace_destroy(s->ws[i]);
  }
  if (s->arena) cudaFree(s->arena);
  if (s->d_segs) cudaFree(s->d_segs);
  if (s->h_segs) cudaFreeHost(s->h_segs);
  delete s;
}

}  // extern "C"
