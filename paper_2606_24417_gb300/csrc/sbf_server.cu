// sbf_server.cu -- serving loop for one resident filter (continuous batching).
//
// Clients submit query requests (host reads) from any thread, one at a time
// or many per call.  A worker thread admits queued requests while memory is
// free (admission by memory), coalesces every admitted request into ONE
// launch of the fused query kernel (one segment per request), and keeps up to
// `max_inflight` such launches on separate streams, so requests that arrive
// while others run are admitted and their work overlaps on the device.
//
// Inputs.  On a GB300 the GPU reads host memory over NVLink-C2C: pinned
// (page-locked, mapped) buffers always, and ordinary pageable buffers when the
// device reads them through the host's page tables (address translation
// services).  A request whose bytes and offsets the device can read this way
// is read in place by the kernel -- no copy, no per-request API call; its
// bytes still count against the read budget while it is in flight.  Other
// requests are copied into a device read arena first (the staged path, also
// forced by SBF_SERVER_STAGE_INPUTS).
//
// Results.  Hit counts (and answer words when asked for) land in a device
// result arena, go back to a pinned mirror with one copy per contiguous run
// of the launch's result regions, and are copied to the callers' buffers by
// the worker after the launch completes, outside the lock.
//
// Every host wait is bounded (timeouts); nothing on the device waits.
// Scheduling never changes the answers: each request gets exactly the bits
// and hit counts of a sbf_query_seqs call on its own reads.
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
    if (n == 0) {
      *at = 0;
      return true;
    }
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
    if (n == 0) return;
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
  // device-visible views of the inputs (direct reads), or NULL: staged
  const uint8_t* v_seq = nullptr;
  const uint64_t* v_off = nullptr;
  uint64_t seq_at = 0, seq_bytes = 0;    // staged reads in the read arena
  uint64_t off_at = 0, off_bytes = 0;    // staged offsets in the offset arena
  uint64_t budget_bytes = 0;             // read bytes counted against the budget
  uint64_t res_at = 0, res_bytes = 0;    // hits, then answer words, in the result arena
  uint64_t bits_at = 0;                  // answer words' place in the result arena
  uint64_t kmers = 0;
  Clock::time_point t_submit, t_admit, t_launch, t_complete, t_done;
  int state = 0;                         // 0 queued, 1 in flight, 2 done, < 0 error code
};

struct Launch {
  std::vector<Request*> reqs;
  int slot = 0;
  uint64_t seq_used = 0;                 // budget bytes of direct requests
};

// Zeroes each segment's hit counts and answer words (when it has them) before
// the query: one launch for a whole batch of requests.  Block b handles
// segments b, b + gridDim.x, ...
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

constexpr int kStages = 4;   // queue, launch, device, delivery

}  // namespace

struct sbf_server {
  const sbf_filter* filter = nullptr;
  int device = 0;
  int max_inflight = 2;
  uint32_t max_per_launch = 4096;
  bool stage_inputs = false;        // SBF_SERVER_STAGE_INPUTS
  bool pageable_direct = false;     // the device reads pageable memory via host page tables
  // device arenas: staged reads and offsets; results (hits and answer words)
  uint8_t* d_seq = nullptr;
  uint8_t* d_off = nullptr;
  uint8_t* d_res = nullptr;
  uint8_t* h_res = nullptr;         // pinned mirror of the result arena
  std::unique_ptr<Arena> seq_arena, off_arena, res_arena;
  uint64_t read_budget = 0, direct_in_flight = 0;
  // read bytes after which a launch takes no further request, so that a deep
  // queue becomes several launches whose result copies and delivery overlap
  // the next launch's kernel
  uint64_t launch_cap = 0;
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
  std::vector<double> stage_s[kStages];
  uint64_t kmers_done = 0, launches = 0, direct_reqs = 0, staged_reqs = 0;
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

// The address through which the device reads host memory p, or NULL if it
// cannot: page-locked memory mapped into the device's address space, or any
// host memory when the device reads pageable memory through the host's page
// tables.
const void* device_view(const sbf_server* s, const void* p) {
  if (!p) return nullptr;
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (a.type == cudaMemoryTypeHost) return a.devicePointer;  // NULL if not mapped for this device
  if (a.type == cudaMemoryTypeUnregistered && s->pageable_direct) return p;
  return nullptr;
}

// Place one request: device views of its inputs (or arena space to stage
// them) and result space.  Caller holds s->mu.  False: no room yet.
bool admit(sbf_server* s, Request* r, Launch& L) {
  const bool direct = r->v_seq && (r->v_off || r->n_reads == 0);
  uint64_t sa = 0, oa = 0, ra = 0;
  if (direct) {
    // read in place: only the budget of read bytes in flight applies
    if (s->direct_in_flight + L.seq_used + r->budget_bytes > s->read_budget) return false;
  } else {
    if (!s->seq_arena->alloc(r->seq_bytes, 32, &sa)) return false;
    if (!s->off_arena->alloc(r->off_bytes, 16, &oa)) {
      s->seq_arena->release(sa, r->seq_bytes);
      return false;
    }
  }
  if (!s->res_arena->alloc(r->res_bytes, 16, &ra)) {
    if (!direct) {
      s->seq_arena->release(sa, r->seq_bytes);
      s->off_arena->release(oa, r->off_bytes);
    }
    return false;
  }
  if (direct) {
    L.seq_used += r->budget_bytes;
    r->seq_bytes = r->off_bytes = 0;
  } else {
    r->v_seq = nullptr;
    r->v_off = nullptr;
    r->seq_at = sa;
    r->off_at = oa;
  }
  r->res_at = ra;
  r->bits_at = ra + (r->n_reads * 4 + 15) / 16 * 16;
  return true;
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
    const uint8_t* seq = r->v_seq;
    const uint64_t* off = r->v_off;
    if (!seq) {  // staged: copy the request's bytes and offsets into the arenas
      seq = s->d_seq + r->seq_at;
      off = reinterpret_cast<const uint64_t*>(s->d_off + r->off_at);
      if ((r->seq_len &&
           (e = cudaMemcpyAsync(s->d_seq + r->seq_at, r->h_seq, r->seq_len, cudaMemcpyHostToDevice,
                                st)) != cudaSuccess) ||
          (e = cudaMemcpyAsync(s->d_off + r->off_at, r->h_off, (r->n_reads + 1) * 8,
                               cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return cuda_fail(e, "server staging");
    }
    Segment sg{};
    sg.words = g.words;
    sg.n_shards = g.n_shards;
    sg.seq = seq;                    // the request's own bytes, offsets as submitted
    sg.seq_len = r->seq_len;
    sg.off = off;
    sg.n_reads = r->n_reads;
    sg.bits = r->h_bits ? reinterpret_cast<uint32_t*>(s->d_res + r->bits_at) : nullptr;
    sg.hits = reinterpret_cast<uint32_t*>(s->d_res + r->res_at);
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
  // results back to the pinned mirror: one copy per contiguous run of the
  // launch's result regions (consecutive admissions are mostly adjacent)
  std::vector<std::pair<uint64_t, uint64_t>> ranges;
  ranges.reserve(L.reqs.size());
  for (const Request* r : L.reqs) {
    const uint64_t used = r->h_bits ? r->res_bytes : r->n_reads * 4;
    if (used) ranges.emplace_back(r->res_at, r->res_at + used);
  }
  std::sort(ranges.begin(), ranges.end());
  for (size_t i = 0; i < ranges.size();) {
    uint64_t a = ranges[i].first, b = ranges[i].second;
    size_t j = i + 1;
    // merge regions whose gap is small (alignment padding or a few bytes)
    while (j < ranges.size() && ranges[j].first <= b + 256) {
      b = std::max(b, ranges[j].second);
      ++j;
    }
    if ((e = cudaMemcpyAsync(s->h_res + a, s->d_res + a, b - a, cudaMemcpyDeviceToHost, st)) !=
        cudaSuccess)
      return cuda_fail(e, "server results");
    i = j;
  }
  if ((e = cudaEventRecord(s->events[slot], st)) != cudaSuccess) return cuda_fail(e, "server event");
  // wake the worker when this launch's work is done instead of letting it poll
  if ((e = cudaLaunchHostFunc(st, on_launch_done, s)) != cudaSuccess)
    return cuda_fail(e, "server completion callback");
  return SBF_OK;
}

// Copy a finished launch's results from the pinned mirror to the callers'
// buffers (no lock needed: the requests' arena space is still theirs).
void deliver(sbf_server* s, const Launch& L) {
  for (const Request* r : L.reqs) {
    if (r->h_hits && r->n_reads) std::memcpy(r->h_hits, s->h_res + r->res_at, r->n_reads * 4);
    if (r->h_bits && r->seq_len)
      std::memcpy(r->h_bits, s->h_res + r->bits_at, ((r->seq_len + 31) / 32) * 4);
  }
}

void finish(sbf_server* s, Launch& L, int status) {
  // caller holds s->mu
  const Clock::time_point now = Clock::now();
  s->direct_in_flight -= L.seq_used;
  for (Request* r : L.reqs) {
    r->state = status == SBF_OK ? 2 : status;
    r->t_done = now;
    s->seq_arena->release(r->seq_at, r->seq_bytes);
    s->off_arena->release(r->off_at, r->off_bytes);
    s->res_arena->release(r->res_at, r->res_bytes);
    if (status == SBF_OK) {
      auto d = [](Clock::time_point a, Clock::time_point b) {
        return std::chrono::duration<double>(b - a).count();
      };
      s->latencies.push_back(d(r->t_submit, r->t_done));
      s->stage_s[0].push_back(d(r->t_submit, r->t_admit));
      s->stage_s[1].push_back(d(r->t_admit, r->t_launch));
      s->stage_s[2].push_back(d(r->t_launch, r->t_complete));
      s->stage_s[3].push_back(d(r->t_complete, r->t_done));
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
      const Clock::time_point now = Clock::now();
      for (auto& d : done)
        for (Request* r : d.first.reqs) r->t_complete = now;
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
      const Clock::time_point now = Clock::now();
      uint64_t launch_bytes = 0;
      while (!s->queue.empty() && L.reqs.size() < s->max_per_launch &&
             (L.reqs.empty() || launch_bytes < s->launch_cap)) {
        Request* r = s->queue.front();
        if (!admit(s, r, L)) break;
        launch_bytes += r->budget_bytes;
        r->state = 1;
        r->t_admit = now;
        s->queue.pop_front();
        L.reqs.push_back(r);
        if (r->v_seq) ++s->direct_reqs; else ++s->staged_reqs;
      }
    }
    if (!L.reqs.empty()) {
      L.slot = slot;
      s->slot_busy[slot] = true;
      s->direct_in_flight += L.seq_used;
      ++s->launches;
      lk.unlock();
      int rc = start_launch(s, L);
      const Clock::time_point now = Clock::now();
      lk.lock();
      for (Request* r : L.reqs) r->t_launch = now;
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

// Checks one request and prepares it for the queue (no lock held): offsets,
// k-mer count, the device's view of its inputs and the arena sizes.
int prepare(sbf_server* s, const uint8_t* h_seq, uint64_t seq_len, const uint64_t* h_off,
            uint64_t n_reads, uint32_t* h_read_hits, uint32_t* h_kmer_bits, Request** out) {
  if (!h_off || (seq_len && !h_seq)) return fail(SBF_EINVAL, "bad argument");
  if (h_off[0] != 0 || h_off[n_reads] != seq_len)
    return fail(SBF_EINVAL, "offsets must start at 0 and end at seq_len");
  const int k = s->filter->geom.k;
  uint64_t kmers = 0;
  for (uint64_t i = 0; i < n_reads; ++i) {
    if (h_off[i + 1] < h_off[i])
      return fail(SBF_EINVAL, "offsets decrease at read %llu", (unsigned long long)i);
    const uint64_t len = h_off[i + 1] - h_off[i];
    if (len >= (uint64_t)k) kmers += len - k + 1;
  }
  Request* r = new (std::nothrow) Request();
  if (!r) return fail(SBF_ENOMEM, "host allocation failed");
  r->h_seq = h_seq;
  r->seq_len = seq_len;
  r->h_off = h_off;
  r->n_reads = n_reads;
  r->h_hits = h_read_hits;
  r->h_bits = h_kmer_bits;
  r->kmers = kmers;
  r->seq_bytes = std::max<uint64_t>(32, (seq_len + 31) / 32 * 32);
  r->off_bytes = ((n_reads + 1) * 8 + 15) / 16 * 16;
  r->budget_bytes = r->seq_bytes;
  r->res_bytes = (n_reads * 4 + 15) / 16 * 16 + (h_kmer_bits ? ((seq_len + 31) / 32 * 4 + 15) / 16 * 16 : 0);
  if (r->res_bytes == 0) r->res_bytes = 16;
  if (!s->stage_inputs) {
    r->v_seq = seq_len ? static_cast<const uint8_t*>(device_view(s, h_seq)) : nullptr;
    r->v_off = static_cast<const uint64_t*>(device_view(s, h_off));
    if (!r->v_seq || !r->v_off) r->v_seq = nullptr, r->v_off = nullptr;  // stage both
  }
  if (r->seq_bytes > s->read_budget || r->off_bytes > s->off_arena->size() ||
      r->res_bytes > s->res_arena->size()) {
    delete r;
    return fail(SBF_EINVAL, "request larger than the server's memory budget");
  }
  *out = r;
  return SBF_OK;
}

// Queues prepared requests (one lock for all of them).
void enqueue(sbf_server* s, Request* const* rs, uint64_t n, uint64_t* tickets) {
  const Clock::time_point now = Clock::now();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    for (uint64_t i = 0; i < n; ++i) {
      Request* r = rs[i];
      r->t_submit = now;
      r->id = s->next_id++;
      if (!s->have_first) {
        s->first_submit = now;
        s->have_first = true;
      }
      s->by_id[r->id] = r;
      s->queue.push_back(r);
      tickets[i] = r->id;
    }
    s->submissions += n;
  }
  s->cv_work.notify_one();
}

double percentile(std::vector<double> v, double p) {
  if (v.empty()) return 0.0;
  std::sort(v.begin(), v.end());
  size_t i = (size_t)std::min<double>((double)v.size() - 1, p * (double)(v.size() - 1) + 0.5);
  return v[i];
}

}  // namespace

extern "C" {

int sbf_server_create_ex(const sbf_filter* f, uint64_t read_budget_bytes, int max_inflight,
                         uint32_t max_per_launch, uint32_t flags, sbf_server** out) {
  sbf::clear_error();
  if (!f || !out || read_budget_bytes < 4096 || max_inflight < 1 || max_inflight > 16 ||
      max_per_launch < 1 || max_per_launch > 65536 || (flags & ~(uint32_t)SBF_SERVER_STAGE_INPUTS))
    return fail(SBF_EINVAL, "bad argument");
  *out = nullptr;
  if (!f->fused) return fail(SBF_EUNSUPPORTED, "the server needs a filter with fused kernels");
  sbf_server* s = new (std::nothrow) sbf_server();
  if (!s) return fail(SBF_ENOMEM, "host allocation failed");
  s->filter = f;
  s->device = f->device;
  s->max_inflight = max_inflight;
  s->max_per_launch = max_per_launch;
  s->stage_inputs = (flags & SBF_SERVER_STAGE_INPUTS) != 0;
  const uint64_t seq_bytes = (read_budget_bytes + 31) / 32 * 32;
  s->read_budget = seq_bytes;
  s->launch_cap = std::max<uint64_t>(seq_bytes / (uint64_t)(max_inflight + 1), 1ull << 20);
  // offsets: 8 bytes per read of >= 1 byte is at most 8x the reads; reads of
  // the benchmark's 150 bp need about 1/19 of them.  Results: 4 bytes per
  // read plus one bit per byte.
  const uint64_t off_bytes = seq_bytes / 4 + (1 << 16);
  const uint64_t res_bytes = seq_bytes / 4 + seq_bytes / 8 + (1 << 16);
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(s->device);
  int pageable = 0, host_tables = 0;
  cudaDeviceGetAttribute(&pageable, cudaDevAttrPageableMemoryAccess, s->device);
  cudaDeviceGetAttribute(&host_tables, cudaDevAttrPageableMemoryAccessUsesHostPageTables, s->device);
  s->pageable_direct = pageable == 1 && host_tables == 1;
  bool ok = cudaMalloc(&s->d_seq, seq_bytes) == cudaSuccess &&
            cudaMalloc(&s->d_off, off_bytes) == cudaSuccess &&
            cudaMalloc(&s->d_res, res_bytes) == cudaSuccess &&
            cudaMallocHost(&s->h_res, res_bytes) == cudaSuccess;
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
  s->off_arena.reset(new Arena(off_bytes));
  s->res_arena.reset(new Arena(res_bytes));
  s->worker = std::thread(worker_loop, s);
  *out = s;
  return SBF_OK;
}

int sbf_server_create(const sbf_filter* f, uint64_t read_budget_bytes, int max_inflight,
                      uint32_t max_per_launch, sbf_server** out) {
  return sbf_server_create_ex(f, read_budget_bytes, max_inflight, max_per_launch, 0, out);
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
  cudaFree(s->d_off);
  cudaFree(s->d_res);
  cudaFreeHost(s->h_res);
  cudaSetDevice(prev);
  for (auto& kv : s->by_id) delete kv.second;
  delete s;
}

int sbf_server_submit(sbf_server* s, const uint8_t* h_seq, uint64_t seq_len, const uint64_t* h_off,
                      uint64_t n_reads, uint32_t* h_read_hits, uint32_t* h_kmer_bits,
                      uint64_t* ticket) {
  sbf::clear_error();
  if (!s || !ticket) return fail(SBF_EINVAL, "bad argument");
  // make the device's context current on this thread (a thread that never
  // made a CUDA call has none, and pointer queries would then see no pinned
  // memory)
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(s->device);
  Request* r = nullptr;
  const int rc = prepare(s, h_seq, seq_len, h_off, n_reads, h_read_hits, h_kmer_bits, &r);
  if (prev >= 0 && prev != s->device) cudaSetDevice(prev);
  if (rc != SBF_OK) return rc;
  enqueue(s, &r, 1, ticket);
  return SBF_OK;
}

int sbf_server_submit_batch(sbf_server* s, uint64_t n, const uint8_t* const* h_seqs,
                            const uint64_t* seq_lens, const uint64_t* const* h_offs,
                            const uint64_t* n_reads, uint32_t* const* h_read_hits,
                            uint32_t* const* h_kmer_bits, uint64_t* tickets) {
  sbf::clear_error();
  if (!s || (n && (!h_seqs || !seq_lens || !h_offs || !n_reads || !tickets)))
    return fail(SBF_EINVAL, "bad argument");
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(s->device);
  std::vector<Request*> rs;
  rs.reserve(n);
  int rc = SBF_OK;
  for (uint64_t i = 0; i < n && rc == SBF_OK; ++i) {
    Request* r = nullptr;
    rc = prepare(s, h_seqs[i], seq_lens[i], h_offs[i], n_reads[i],
                 h_read_hits ? h_read_hits[i] : nullptr, h_kmer_bits ? h_kmer_bits[i] : nullptr, &r);
    if (rc == SBF_OK) rs.push_back(r);
  }
  if (prev >= 0 && prev != s->device) cudaSetDevice(prev);
  if (rc != SBF_OK) {  // nothing is queued when any request is refused
    for (Request* r : rs) delete r;
    return rc;
  }
  enqueue(s, rs.data(), n, tickets);
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
  const std::vector<double>& v = s->latencies;
  if (completed) *completed = v.size();
  if (p50_s) *p50_s = percentile(v, 0.50);
  if (p99_s) *p99_s = percentile(v, 0.99);
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

int sbf_server_breakdown(sbf_server* s, double* p50_s, double* p99_s, uint64_t* direct,
                         uint64_t* staged) {
  sbf::clear_error();
  if (!s) return fail(SBF_EINVAL, "server is NULL");
  std::lock_guard<std::mutex> lk(s->mu);
  for (int i = 0; i < kStages; ++i) {
    if (p50_s) p50_s[i] = percentile(s->stage_s[i], 0.50);
    if (p99_s) p99_s[i] = percentile(s->stage_s[i], 0.99);
  }
  if (direct) *direct = s->direct_reqs;
  if (staged) *staged = s->staged_reqs;
  return SBF_OK;
}

int sbf_server_reset_stats(sbf_server* s) {
  sbf::clear_error();
  if (!s) return fail(SBF_EINVAL, "server is NULL");
  std::lock_guard<std::mutex> lk(s->mu);
  s->latencies.clear();
  for (auto& v : s->stage_s) v.clear();
  s->kmers_done = 0;
  s->launches = 0;
  s->direct_reqs = s->staged_reqs = 0;
  s->have_first = false;
  return SBF_OK;
}

}  // extern "C"
