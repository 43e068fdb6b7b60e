// sbf_server.cu -- serving loop for one resident filter (continuous batching).
//
// Clients submit query requests (host reads) from any thread.  A worker
// thread admits queued requests while device memory for their reads, offsets
// and hit counts is free in a fixed arena (admission by memory), coalesces
// every admitted request into ONE launch of the fused query kernel (one
// segment per request), and keeps up to `max_inflight` such launches on
// separate streams so that requests arriving while others run are admitted
// and their copies and kernels overlap on the device.  A launch completes
// when its event fires; its requests' device memory is then freed.  Every
// host wait is bounded (timeouts); nothing on the device waits.  Scheduling
// never changes the answers: each request gets exactly the bits and hit
// counts of a sbf_query_seqs call on its own reads.
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
#include <unordered_map>
#include <vector>

#include "sbf_fused.cuh"

using sbf::fused::Params;
using sbf::fused::Segment;
using Clock = std::chrono::steady_clock;

namespace {

// First-fit allocator over [0, size) with coalescing frees.
class Arena {
 public:
  explicit Arena(uint64_t size) : size_(size) { free_[0] = size; }
  bool alloc(uint64_t n, uint64_t align, uint64_t* at) {
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      uint64_t start = (it->first + align - 1) / align * align;
      uint64_t end = it->first + it->second;
      if (start + n <= end) {
        uint64_t f0 = it->first, f1 = end;
        free_.erase(it);
        if (start > f0) free_[f0] = start - f0;
        if (start + n < f1) free_[start + n] = f1 - (start + n);
        *at = start;
        return true;
      }
    }
    return false;
  }
  void release(uint64_t at, uint64_t n) {
    auto it = free_.emplace(at, n).first;
    auto next = std::next(it);
    if (next != free_.end() && it->first + it->second == next->first) {
      it->second += next->second;
      free_.erase(next);
    }
    if (it != free_.begin()) {
      auto prev = std::prev(it);
      if (prev->first + prev->second == it->first) {
        prev->second += it->second;
        free_.erase(it);
      }
    }
  }
  uint64_t size() const { return size_; }

 private:
  uint64_t size_;
  std::map<uint64_t, uint64_t> free_;
};

struct Request {
  uint64_t id = 0;
  const uint8_t* h_seq = nullptr;
  uint64_t seq_len = 0;
  const uint64_t* h_off = nullptr;
  uint64_t n_reads = 0;
  uint32_t* h_hits = nullptr;
  uint32_t* h_bits = nullptr;
  uint64_t seq_at = 0, seq_bytes = 0;    // placement in the read arena
  uint64_t meta_at = 0, meta_bytes = 0;  // offsets + hits in the meta arena
  uint64_t kmers = 0;
  Clock::time_point t_submit, t_done;
  int state = 0;                         // 0 queued, 1 in flight, 2 done, < 0 error code
};

struct Launch {
  std::vector<Request*> reqs;
  int slot = 0;
};

// Zeroes each segment's hit counts and answer words (when it has them) before
// the query: one launch for a whole batch of requests instead of two memsets
// per request.  Block b handles segments b, b + gridDim.x, ...
__global__ void zero_segments(const Segment* __restrict__ segs, uint32_t n_segs) {
  for (uint32_t i = blockIdx.x; i < n_segs; i += gridDim.x) {
    const Segment sg = segs[i];
    for (uint64_t j = threadIdx.x; j < sg.n_reads; j += blockDim.x) sg.hits[j] = 0u;
    if (sg.bits) {
      const uint64_t nw = (sg.seq_len + 31) / 32;
      for (uint64_t j = threadIdx.x; j < nw; j += blockDim.x) sg.bits[j] = 0u;
    }
  }
}

}  // namespace

struct sbf_server {
  const sbf_filter* filter = nullptr;
  int device = 0;
  int max_inflight = 2;
  uint32_t max_per_launch = 4096;
  // device arenas
  uint8_t* d_seq = nullptr;     // reads
  uint32_t* d_bits = nullptr;   // answers, one bit per read-arena byte
  uint8_t* d_meta = nullptr;    // offsets and hit counts
  // pinned host mirrors of the result arenas: results land here
  // asynchronously and are copied to the caller's buffers after completion
  // (a device-to-host copy into pageable memory would block the worker)
  uint8_t* h_meta = nullptr;
  uint32_t* h_bits = nullptr;
  std::unique_ptr<Arena> seq_arena, meta_arena;
  // per launch slot: stream, event, segment tables
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> events;
  std::vector<Segment*> h_tables, d_tables;
  std::vector<bool> slot_busy;
  // queue and bookkeeping
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request*> queue;
  std::unordered_map<uint64_t, Request*> by_id;
  std::vector<Launch> inflight;
  uint64_t next_id = 1;
  uint64_t completions = 0;     // launches whose stream work has finished (host callbacks)
  uint64_t submissions = 0;     // requests submitted so far
  bool stop = false;
  std::thread worker;
  // statistics
  std::vector<double> latencies;
  uint64_t kmers_done = 0, launches = 0;
  Clock::time_point first_submit, last_done;
  bool have_first = false;
};

namespace {

using sbf::cuda_fail;
using sbf::fail;

// Runs on a CUDA callback thread once a launch's stream work is done: counts
// the completion and wakes the worker (no CUDA calls allowed here).
void CUDART_CB on_launch_done(void* arg) {
  sbf_server* s = static_cast<sbf_server*>(arg);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    ++s->completions;
  }
  s->cv_work.notify_all();
}

// Launch every request of `L` as one segment each, on slot L.slot.
int start_launch(sbf_server* s, Launch& L) {
  const sbf::Geom& g = s->filter->geom;
  const int slot = L.slot;
  cudaStream_t st = s->streams[slot];
  const uint64_t adv = (uint64_t)sbf::fused::advance_of(g);
  Segment* table = s->h_tables[slot];
  uint64_t iters = 0;
  cudaError_t e = cudaSuccess;
  for (size_t i = 0; i < L.reqs.size(); ++i) {
    Request* r = L.reqs[i];
    uint64_t* d_off = reinterpret_cast<uint64_t*>(s->d_meta + r->meta_at);
    uint32_t* d_hits = reinterpret_cast<uint32_t*>(d_off + r->n_reads + 1);
    if ((e = cudaMemcpyAsync(s->d_seq + r->seq_at, r->h_seq, r->seq_len, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(d_off, r->h_off, (r->n_reads + 1) * 8, cudaMemcpyHostToDevice, st)) != cudaSuccess)
      return cuda_fail(e, "server staging");
    Segment sg{};
    sg.words = g.words;
    sg.n_shards = g.n_shards;
    sg.seq = s->d_seq + r->seq_at;   // the request's own bytes, offsets as submitted
    sg.seq_len = r->seq_len;
    sg.off = d_off;
    sg.n_reads = r->n_reads;
    sg.bits = r->h_bits ? s->d_bits + r->seq_at / 32 : nullptr;  // no answer words wanted: none written
    sg.hits = d_hits;
    sg.p_begin = 0;
    sg.iter_begin = iters;
    sg.iters = (r->seq_len + adv - 1) / adv;
    iters += sg.iters;
    table[i] = sg;
  }
  if ((e = cudaMemcpyAsync(s->d_tables[slot], table, L.reqs.size() * sizeof(Segment),
                           cudaMemcpyHostToDevice, st)) != cudaSuccess)
    return cuda_fail(e, "server table upload");
  {
    const uint32_t n = (uint32_t)L.reqs.size();
    zero_segments<<<n < 1024u ? n : 1024u, 256, 0, st>>>(s->d_tables[slot], n);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "server zeroing");
  }
  Params P{};
  P.g = g;
  P.stats = nullptr;
  P.segs = s->d_tables[slot];
  P.n_segs = (uint32_t)L.reqs.size();
  P.iters = iters;
  P.work = nullptr;
  P.chunk = 1;
  P.grid_blocks = 0;
  P.big = sbf::fused::is_big(g) ? 1u : 0u;
  if ((e = sbf::fused::launch_params(P, false, st)) != cudaSuccess) return cuda_fail(e, "server launch");
  for (Request* r : L.reqs) {
    const uint64_t hits_at = r->meta_at + (r->n_reads + 1) * 8;
    if (r->h_hits && r->n_reads &&
        (e = cudaMemcpyAsync(s->h_meta + hits_at, s->d_meta + hits_at, r->n_reads * 4,
                             cudaMemcpyDeviceToHost, st)) != cudaSuccess)
      return cuda_fail(e, "server results");
    if (r->h_bits && r->seq_len &&
        (e = cudaMemcpyAsync(s->h_bits + r->seq_at / 32, s->d_bits + r->seq_at / 32,
                             ((r->seq_len + 31) / 32) * 4, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
      return cuda_fail(e, "server results");
  }
  if ((e = cudaEventRecord(s->events[slot], st)) != cudaSuccess) return cuda_fail(e, "server event");
  // wake the worker when this launch's work is done instead of letting it poll
  if ((e = cudaLaunchHostFunc(st, on_launch_done, s)) != cudaSuccess)
    return cuda_fail(e, "server completion callback");
  return SBF_OK;
}

// Copy a finished launch's results from the pinned mirrors to the callers'
// buffers (no lock needed: the requests' arena space is still theirs).
void deliver(sbf_server* s, const Launch& L) {
  for (const Request* r : L.reqs) {
    if (r->h_hits && r->n_reads)
      std::memcpy(r->h_hits, s->h_meta + r->meta_at + (r->n_reads + 1) * 8, r->n_reads * 4);
    if (r->h_bits && r->seq_len)
      std::memcpy(r->h_bits, s->h_bits + r->seq_at / 32, ((r->seq_len + 31) / 32) * 4);
  }
}

void finish(sbf_server* s, Launch& L, int status) {
  // caller holds s->mu
  const Clock::time_point now = Clock::now();
  for (Request* r : L.reqs) {
    r->state = status == SBF_OK ? 2 : status;
    r->t_done = now;
    s->seq_arena->release(r->seq_at, r->seq_bytes);
    s->meta_arena->release(r->meta_at, r->meta_bytes);
    if (status == SBF_OK) {
      s->latencies.push_back(std::chrono::duration<double>(r->t_done - r->t_submit).count());
      s->kmers_done += r->kmers;
      s->last_done = now;
    }
  }
  s->slot_busy[L.slot] = false;
}

void worker_loop(sbf_server* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  while (true) {
    // retire finished launches: results are copied out without the lock
    std::vector<std::pair<Launch, int>> done;
    for (size_t i = 0; i < s->inflight.size();) {
      cudaError_t q = cudaEventQuery(s->events[s->inflight[i].slot]);
      if (q == cudaErrorNotReady) {
        ++i;
        continue;
      }
      done.emplace_back(std::move(s->inflight[i]), q == cudaSuccess ? SBF_OK : SBF_ECUDA);
      s->inflight.erase(s->inflight.begin() + i);
    }
    if (!done.empty()) {
      lk.unlock();
      for (auto& d : done)
        if (d.second == SBF_OK) deliver(s, d.first);
      lk.lock();
      for (auto& d : done) finish(s, d.first, d.second);
      s->cv_done.notify_all();
    }
    if (s->stop && s->queue.empty() && s->inflight.empty()) break;
    // admit queued requests into the next launch while memory and a slot allow
    int slot = -1;
    for (int i = 0; i < s->max_inflight; ++i)
      if (!s->slot_busy[i]) {
        slot = i;
        break;
      }
    Launch L;
    if (slot >= 0) {
      while (!s->queue.empty() && L.reqs.size() < s->max_per_launch) {
        Request* r = s->queue.front();
        uint64_t sa = 0, ma = 0;
        if (!s->seq_arena->alloc(r->seq_bytes, 32, &sa)) break;
        if (!s->meta_arena->alloc(r->meta_bytes, 16, &ma)) {
          s->seq_arena->release(sa, r->seq_bytes);
          break;
        }
        r->seq_at = sa;
        r->meta_at = ma;
        r->state = 1;
        s->queue.pop_front();
        L.reqs.push_back(r);
      }
    }
    if (!L.reqs.empty()) {
      L.slot = slot;
      s->slot_busy[slot] = true;
      ++s->launches;
      lk.unlock();
      int rc = start_launch(s, L);
      lk.lock();
      if (rc != SBF_OK) {
        finish(s, L, rc);
        s->cv_done.notify_all();
      } else {
        s->inflight.push_back(std::move(L));
      }
      continue;
    }
    // nothing to admit: wait for a submission or a completion callback (the
    // timeout only bounds the wait; callbacks and submissions notify)
    const uint64_t seen_c = s->completions, seen_s = s->submissions;
    s->cv_work.wait_for(lk, std::chrono::milliseconds(s->inflight.empty() ? 5 : 1), [&] {
      return s->completions != seen_c || s->submissions != seen_s || s->stop;
    });
  }
}

}  // namespace

extern "C" {

int sbf_server_create(const sbf_filter* f, uint64_t read_budget_bytes, int max_inflight,
                      uint32_t max_per_launch, sbf_server** out) {
  sbf::clear_error();
  if (!f || !out || read_budget_bytes < 4096 || max_inflight < 1 || max_inflight > 16 ||
      max_per_launch < 1 || max_per_launch > 65536)
    return fail(SBF_EINVAL, "bad argument");
  *out = nullptr;
  if (!f->fused) return fail(SBF_EUNSUPPORTED, "the server needs a filter with fused kernels");
  sbf_server* s = new (std::nothrow) sbf_server();
  if (!s) return fail(SBF_ENOMEM, "host allocation failed");
  s->filter = f;
  s->device = f->device;
  s->max_inflight = max_inflight;
  s->max_per_launch = max_per_launch;
  const uint64_t seq_bytes = (read_budget_bytes + 31) / 32 * 32;
  const uint64_t meta_bytes = seq_bytes / 4 + (1 << 16);
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(s->device);
  bool ok = cudaMalloc(&s->d_seq, seq_bytes) == cudaSuccess &&
            cudaMalloc(&s->d_bits, seq_bytes / 8) == cudaSuccess &&
            cudaMalloc(&s->d_meta, meta_bytes) == cudaSuccess &&
            cudaMallocHost(&s->h_bits, seq_bytes / 8) == cudaSuccess &&
            cudaMallocHost(&s->h_meta, meta_bytes) == cudaSuccess;
  s->streams.resize(max_inflight);
  s->events.resize(max_inflight);
  s->h_tables.resize(max_inflight);
  s->d_tables.resize(max_inflight);
  s->slot_busy.assign(max_inflight, false);
  for (int i = 0; ok && i < max_inflight; ++i) {
    ok = cudaStreamCreateWithFlags(&s->streams[i], cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&s->events[i], cudaEventDisableTiming) == cudaSuccess &&
         cudaMallocHost(&s->h_tables[i], s->max_per_launch * sizeof(Segment)) == cudaSuccess &&
         cudaMalloc(&s->d_tables[i], s->max_per_launch * sizeof(Segment)) == cudaSuccess;
  }
  // initialise the kernel's attributes before the worker launches it
  if (ok) {
    Params P{};
    P.g = f->geom;
    P.big = sbf::fused::is_big(f->geom) ? 1u : 0u;
    ok = sbf::fused::launch_params(P, false, s->streams[0]) == cudaSuccess;
  }
  cudaSetDevice(prev);
  if (!ok) {
    cudaGetLastError();
    sbf_server_destroy(s);
    return fail(SBF_ENOMEM, "server device allocation failed");
  }
  s->seq_arena.reset(new Arena(seq_bytes));
  s->meta_arena.reset(new Arena(meta_bytes));
  s->worker = std::thread(worker_loop, s);
  *out = s;
  return SBF_OK;
}

void sbf_server_destroy(sbf_server* s) {
  if (!s) return;
  if (s->worker.joinable()) {
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->stop = true;
    }
    s->cv_work.notify_all();
    s->worker.join();
  }
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(s->device);
  for (size_t i = 0; i < s->streams.size(); ++i) {
    if (s->streams[i]) cudaStreamSynchronize(s->streams[i]);
    if (s->streams[i]) cudaStreamDestroy(s->streams[i]);
    if (s->events[i]) cudaEventDestroy(s->events[i]);
    if (s->h_tables[i]) cudaFreeHost(s->h_tables[i]);
    if (s->d_tables[i]) cudaFree(s->d_tables[i]);
  }
  cudaFree(s->d_seq);
  cudaFree(s->d_bits);
  cudaFree(s->d_meta);
  cudaFreeHost(s->h_bits);
  cudaFreeHost(s->h_meta);
  cudaSetDevice(prev);
  for (auto& kv : s->by_id) delete kv.second;
  delete s;
}

int sbf_server_submit(sbf_server* s, const uint8_t* h_seq, uint64_t seq_len, const uint64_t* h_off,
                      uint64_t n_reads, uint32_t* h_read_hits, uint32_t* h_kmer_bits,
                      uint64_t* ticket) {
  sbf::clear_error();
  if (!s || !ticket || !h_off || (seq_len && !h_seq)) return fail(SBF_EINVAL, "bad argument");
  if (h_off[0] != 0 || h_off[n_reads] != seq_len)
    return fail(SBF_EINVAL, "offsets must start at 0 and end at seq_len");
  for (uint64_t r = 0; r < n_reads; ++r)
    if (h_off[r + 1] < h_off[r]) return fail(SBF_EINVAL, "offsets decrease at read %llu", (unsigned long long)r);
  Request* r = new (std::nothrow) Request();
  if (!r) return fail(SBF_ENOMEM, "host allocation failed");
  r->h_seq = h_seq;
  r->seq_len = seq_len;
  r->h_off = h_off;
  r->n_reads = n_reads;
  r->h_hits = h_read_hits;
  r->h_bits = h_kmer_bits;
  r->seq_bytes = std::max<uint64_t>(32, (seq_len + 31) / 32 * 32);
  r->meta_bytes = ((n_reads + 1) * 8 + n_reads * 4 + 15) / 16 * 16;
  const int k = s->filter->geom.k;
  for (uint64_t i = 0; i < n_reads; ++i) {
    uint64_t len = h_off[i + 1] - h_off[i];
    if (len >= (uint64_t)k) r->kmers += len - k + 1;
  }
  if (r->seq_bytes > s->seq_arena->size() || r->meta_bytes > s->meta_arena->size()) {
    delete r;
    return fail(SBF_EINVAL, "request larger than the server's memory budget");
  }
  r->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    r->id = s->next_id++;
    if (!s->have_first) {
      s->first_submit = r->t_submit;
      s->have_first = true;
    }
    s->by_id[r->id] = r;
    s->queue.push_back(r);
    ++s->submissions;
    *ticket = r->id;
  }
  s->cv_work.notify_one();
  return SBF_OK;
}

int sbf_server_wait(sbf_server* s, uint64_t ticket, double timeout_s, double* latency_s) {
  sbf::clear_error();
  if (!s) return fail(SBF_EINVAL, "server is NULL");
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->by_id.find(ticket);
  if (it == s->by_id.end()) return fail(SBF_EINVAL, "unknown ticket %llu", (unsigned long long)ticket);
  Request* r = it->second;
  const auto deadline = Clock::now() + std::chrono::duration_cast<Clock::duration>(
                                           std::chrono::duration<double>(timeout_s));
  while (r->state == 0 || r->state == 1) {
    if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout &&
        (r->state == 0 || r->state == 1))
      return fail(SBF_ETIMEOUT, "request %llu not done after %.3f s", (unsigned long long)ticket, timeout_s);
  }
  const int st = r->state;
  if (latency_s) *latency_s = std::chrono::duration<double>(r->t_done - r->t_submit).count();
  s->by_id.erase(it);
  delete r;
  return st == 2 ? SBF_OK : fail(st, "request failed on the device");
}

int sbf_server_stats(sbf_server* s, uint64_t* completed, double* p50_s, double* p99_s,
                     double* mean_s, double* kmers_per_s, uint64_t* launches) {
  sbf::clear_error();
  if (!s) return fail(SBF_EINVAL, "server is NULL");
  std::lock_guard<std::mutex> lk(s->mu);
  std::vector<double> v = s->latencies;
  std::sort(v.begin(), v.end());
  auto pct = [&](double p) -> double {
    if (v.empty()) return 0.0;
    size_t i = (size_t)std::min<double>((double)v.size() - 1, p * (double)(v.size() - 1) + 0.5);
    return v[i];
  };
  if (completed) *completed = v.size();
  if (p50_s) *p50_s = pct(0.50);
  if (p99_s) *p99_s = pct(0.99);
  if (mean_s) {
    double sum = 0;
    for (double x : v) sum += x;
    *mean_s = v.empty() ? 0.0 : sum / (double)v.size();
  }
  if (kmers_per_s) {
    double span = s->have_first ? std::chrono::duration<double>(s->last_done - s->first_submit).count() : 0;
    *kmers_per_s = span > 0 ? (double)s->kmers_done / span : 0.0;
  }
  if (launches) *launches = s->launches;
  return SBF_OK;
}

int sbf_server_reset_stats(sbf_server* s) {
  sbf::clear_error();
  if (!s) return fail(SBF_EINVAL, "server is NULL");
  std::lock_guard<std::mutex> lk(s->mu);
  s->latencies.clear();
  s->kmers_done = 0;
  s->launches = 0;
  s->have_first = false;
  return SBF_OK;
}

}  // extern "C"
