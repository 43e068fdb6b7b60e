// sbf_fastx_gpu.cu -- FASTA / FASTQ tokenising on the device.
//
// The host only moves raw text: a chunk of whole records is copied to the
// device (over NVLink-C2C on GB300) and turned there into a read batch --
// the sequence bytes of every record back to back and one offset per record
// -- that the insert and query kernels take directly.  The rules are those of
// the host parser (sbf_fastx.cu) for the inputs it accepts:
//  * FASTA: a record is a line starting with '>' and the lines up to the next
//    such line; its sequence is those lines without '\n', '\r', ' ', '\t'.
//  * FASTQ with four-line records: '@' header, one sequence line, '+' line,
//    one quality line of as many bytes as the sequence has.
// Anything else -- a FASTA line starting with '@', a FASTQ record that is not
// four lines, a quality line of another length -- sets an error flag, and the
// caller parses that chunk on the host instead.
//
// Three passes over 4 KB tiles (256 threads x 16 bytes) with a scan over the
// tiles between them: (A) newlines and the last line start of each tile;
// (B) each byte's line index and line start give its line's role, hence
// which bytes are kept and where records start, counted per tile (and the
// newline positions are written); (C) the kept bytes are compacted and each
// record's offset written.  A last kernel checks FASTQ quality lengths.
#include <cstring>

#include "sbf_internal.h"

namespace {

using sbf::cuda_fail;
using sbf::fail;

constexpr int kTpb = 256;                 // threads per tile
constexpr int kBpt = 16;                  // bytes per thread
constexpr uint64_t kTile = kTpb * kBpt;   // 4096 bytes

__device__ __forceinline__ bool is_blank(uint32_t c) {
  return c == '\n' || c == '\r' || c == ' ' || c == '\t';
}

// Block-wide exclusive scans over 256 threads (sum and max).
__device__ __forceinline__ uint32_t block_excl_sum(uint32_t v, uint32_t* sh, uint32_t* total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, d);
    if (lane >= d) x += y;
  }
  if (lane == 31) sh[w] = x;
  __syncthreads();
  if (w == 0) {
    uint32_t t = lane < kTpb / 32 ? sh[lane] : 0u;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, t, d);
      if (lane >= d) t += y;
    }
    if (lane < kTpb / 32) sh[lane] = t;
  }
  __syncthreads();
  const uint32_t before = (w ? sh[w - 1] : 0u) + x - v;
  if (total) *total = sh[kTpb / 32 - 1];
  __syncthreads();
  return before;
}

__device__ __forceinline__ int64_t block_excl_max(int64_t v, int64_t* sh) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int64_t x = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int64_t y = __shfl_up_sync(0xFFFFFFFFu, x, d);
    if (lane >= d && y > x) x = y;
  }
  const int64_t excl_in_warp = __shfl_up_sync(0xFFFFFFFFu, x, 1);
  if (lane == 31) sh[w] = x;
  __syncthreads();
  if (w == 0) {
    int64_t t = lane < kTpb / 32 ? sh[lane] : -1;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int64_t y = __shfl_up_sync(0xFFFFFFFFu, t, d);
      if (lane >= d && y > t) t = y;
    }
    if (lane < kTpb / 32) sh[lane] = t;
  }
  __syncthreads();
  int64_t before = w ? sh[w - 1] : -1;
  if (lane > 0 && excl_in_warp > before) before = excl_in_warp;
  __syncthreads();
  return before;
}

struct Bytes16 {
  uint8_t b[kBpt];
};

__device__ __forceinline__ Bytes16 load_bytes(const uint8_t* text, uint64_t len, uint64_t p0) {
  Bytes16 r;
  if (p0 + kBpt <= len) {
    const uint4 v = *reinterpret_cast<const uint4*>(text + p0);
    std::memcpy(r.b, &v, kBpt);
  } else {
#pragma unroll
    for (int i = 0; i < kBpt; ++i) r.b[i] = p0 + i < len ? text[p0 + i] : 0;
  }
  return r;
}

// (A) per tile: newlines, and the last line start (-1 if none).
__global__ void __launch_bounds__(kTpb) pass_a(const uint8_t* __restrict__ text, uint64_t len,
                                                uint32_t* tile_nl, int64_t* tile_ls) {
  __shared__ uint32_t sh[32];
  __shared__ int64_t shm[32];
  const uint64_t p0 = blockIdx.x * kTile + (uint64_t)threadIdx.x * kBpt;
  const Bytes16 x = load_bytes(text, len, p0);
  uint32_t prev = p0 == 0 ? '\n' : (p0 <= len ? text[p0 - 1] : 0);
  uint32_t nl = 0;
  int64_t ls = -1;
#pragma unroll
  for (int i = 0; i < kBpt; ++i) {
    const uint64_t p = p0 + i;
    if (p < len) {
      if (prev == '\n') ls = (int64_t)p;
      nl += x.b[i] == '\n';
    }
    prev = x.b[i];
  }
  uint32_t total = 0;
  block_excl_sum(nl, sh, &total);
  const int64_t before = block_excl_max(ls, shm);
  if (threadIdx.x == kTpb - 1) {
    tile_nl[blockIdx.x] = total;
    tile_ls[blockIdx.x] = ls > before ? ls : before;
  }
}

// Exclusive scans over the tiles: two sums (u32 counts -> u64 bases) and one
// max (i64), in three kernels: totals of 1024-tile groups, a scan of the
// group totals (one block), and a scan inside each group from its base.
constexpr int kScan = 1024;

struct ScanIO {
  const uint32_t* a;   // counts to sum (or NULL)
  const uint32_t* b;
  const int64_t* m;    // values to max (or NULL)
  uint64_t* a_out;     // exclusive bases
  uint64_t* b_out;
  int64_t* m_out;
  uint64_t* ga;        // group totals / bases
  uint64_t* gb;
  int64_t* gm;
  uint64_t n;
  uint64_t* totals;    // [0] sum of a, [1] sum of b (written by the top scan)
};

__device__ __forceinline__ void block_scan3(uint64_t& a, uint64_t& b, int64_t& m, uint64_t* sa,
                                            uint64_t* sb, int64_t* sm) {
  // inclusive block scan (Hillis-Steele over shared memory) of 1024 values
  sa[threadIdx.x] = a;
  sb[threadIdx.x] = b;
  sm[threadIdx.x] = m;
  __syncthreads();
  for (int d = 1; d < kScan; d <<= 1) {
    uint64_t ta = 0, tb = 0;
    int64_t tm = -1;
    if ((int)threadIdx.x >= d) {
      ta = sa[threadIdx.x - d];
      tb = sb[threadIdx.x - d];
      tm = sm[threadIdx.x - d];
    }
    __syncthreads();
    sa[threadIdx.x] += ta;
    sb[threadIdx.x] += tb;
    if (tm > sm[threadIdx.x]) sm[threadIdx.x] = tm;
    __syncthreads();
  }
  a = sa[threadIdx.x];
  b = sb[threadIdx.x];
  m = sm[threadIdx.x];
}

__global__ void __launch_bounds__(kScan) scan_groups(ScanIO io) {
  __shared__ uint64_t sa[kScan], sb[kScan];
  __shared__ int64_t sm[kScan];
  const uint64_t i = blockIdx.x * (uint64_t)kScan + threadIdx.x;
  uint64_t a = i < io.n && io.a ? io.a[i] : 0, b = i < io.n && io.b ? io.b[i] : 0;
  int64_t m = i < io.n && io.m ? io.m[i] : -1;
  block_scan3(a, b, m, sa, sb, sm);
  if (threadIdx.x == kScan - 1) {
    io.ga[blockIdx.x] = a;
    io.gb[blockIdx.x] = b;
    io.gm[blockIdx.x] = m;
  }
}

__global__ void __launch_bounds__(kScan) scan_top(ScanIO io, uint64_t groups) {
  __shared__ uint64_t sa[kScan], sb[kScan];
  __shared__ int64_t sm[kScan];
  uint64_t ca = 0, cb = 0;
  int64_t cm = -1;
  for (uint64_t base = 0; base < groups; base += kScan) {
    const uint64_t i = base + threadIdx.x;
    const uint64_t a0 = i < groups ? io.ga[i] : 0, b0 = i < groups ? io.gb[i] : 0;
    const int64_t m0 = i < groups ? io.gm[i] : -1;
    uint64_t a = a0, b = b0;
    int64_t m = m0;
    block_scan3(a, b, m, sa, sb, sm);
    const int64_t m_excl = threadIdx.x ? sm[threadIdx.x - 1] : -1;
    const uint64_t ta = sa[kScan - 1], tb = sb[kScan - 1];
    const int64_t tm = sm[kScan - 1];
    __syncthreads();
    if (i < groups) {
      io.ga[i] = ca + a - a0;
      io.gb[i] = cb + b - b0;
      io.gm[i] = m_excl > cm ? m_excl : cm;
    }
    ca += ta;
    cb += tb;
    if (tm > cm) cm = tm;
    __syncthreads();
  }
  if (threadIdx.x == 0 && io.totals) {
    io.totals[0] = ca;
    io.totals[1] = cb;
  }
}

__global__ void __launch_bounds__(kScan) scan_down(ScanIO io) {
  __shared__ uint64_t sa[kScan], sb[kScan];
  __shared__ int64_t sm[kScan];
  const uint64_t i = blockIdx.x * (uint64_t)kScan + threadIdx.x;
  const uint64_t a0 = i < io.n && io.a ? io.a[i] : 0, b0 = i < io.n && io.b ? io.b[i] : 0;
  const int64_t m0 = i < io.n && io.m ? io.m[i] : -1;
  uint64_t a = a0, b = b0;
  int64_t m = m0;
  block_scan3(a, b, m, sa, sb, sm);
  const int64_t m_excl = threadIdx.x ? sm[threadIdx.x - 1] : -1;
  if (i < io.n) {
    if (io.a_out) io.a_out[i] = io.ga[blockIdx.x] + a - a0;
    if (io.b_out) io.b_out[i] = io.gb[blockIdx.x] + b - b0;
    if (io.m_out) io.m_out[i] = m_excl > io.gm[blockIdx.x] ? m_excl : io.gm[blockIdx.x];
  }
}

cudaError_t scan3(ScanIO io, cudaStream_t st) {
  const uint64_t groups = (io.n + kScan - 1) / kScan;
  scan_groups<<<(int)groups, kScan, 0, st>>>(io);
  scan_top<<<1, kScan, 0, st>>>(io, groups);
  scan_down<<<(int)groups, kScan, 0, st>>>(io);
  return cudaGetLastError();
}

// Per-byte classification shared by passes B and C.
struct ByteInfo {
  uint16_t keep;    // bit i: byte i is a kept sequence byte
  uint16_t rstart;  // bit i: byte i starts a record's header line
  uint16_t nl;      // bit i: byte i is '\n'
  uint32_t bad;     // a line breaks the accepted shapes
};

__device__ __forceinline__ ByteInfo classify(const uint8_t* text, uint64_t len, uint64_t p0,
                                             const Bytes16& x, uint64_t li0, int64_t ls0, int fastq) {
  ByteInfo r{0, 0, 0, 0};
  uint64_t li = li0;   // line index of byte p
  int64_t ls = ls0;    // start of byte p's line
  uint32_t prev = p0 == 0 ? '\n' : (p0 <= len ? text[p0 - 1] : 0);
  uint32_t c0 = ls >= 0 ? text[ls] : 0;  // first byte of the current line
#pragma unroll
  for (int i = 0; i < kBpt; ++i) {
    const uint64_t p = p0 + i;
    const uint32_t c = x.b[i];
    if (p < len) {
      if (prev == '\n') {  // a line starts here
        ls = (int64_t)p;
        c0 = c;
        if (fastq) {
          const uint32_t role = (uint32_t)(li & 3);
          if (role == 0) {
            if (c == '@') r.rstart |= 1u << i; else r.bad = 1;
          } else if (role == 2 && c != '+') {
            r.bad = 1;
          }
        } else {
          if (c == '>') r.rstart |= 1u << i;
          else if (c == '@') r.bad = 1;  // the host parser would start a FASTQ record
        }
      }
      const bool seq_line = fastq ? ((li & 3) == 1) : (c0 != '>');
      if (seq_line && !is_blank(c)) r.keep |= 1u << i;
      if (c == '\n') {
        r.nl |= 1u << i;
        ++li;
      }
    }
    prev = c;
  }
  return r;
}

// (B) per tile: kept bytes and record starts; newline positions.
__global__ void __launch_bounds__(kTpb) pass_b(const uint8_t* __restrict__ text, uint64_t len,
                                                int fastq, const uint64_t* nl_hi,
                                                const int64_t* ls_base,
                                                uint32_t* tile_keep, uint32_t* tile_rec,
                                                uint64_t* line_end, uint32_t* err) {
  __shared__ uint32_t sh[32];
  __shared__ int64_t shm[32];
  const uint64_t p0 = blockIdx.x * kTile + (uint64_t)threadIdx.x * kBpt;
  const Bytes16 x = load_bytes(text, len, p0);
  uint32_t nl = 0;
  int64_t ls = -1;
  uint32_t prev = p0 == 0 ? '\n' : (p0 <= len ? text[p0 - 1] : 0);
#pragma unroll
  for (int i = 0; i < kBpt; ++i) {
    if (p0 + i < len) {
      if (prev == '\n') ls = (int64_t)(p0 + i);
      nl += x.b[i] == '\n';
    }
    prev = x.b[i];
  }
  const uint64_t tile_nl0 = nl_hi[blockIdx.x];
  const uint64_t li0 = tile_nl0 + block_excl_sum(nl, sh, nullptr);
  int64_t ls0 = block_excl_max(ls, shm);
  if (ls_base[blockIdx.x] > ls0) ls0 = ls_base[blockIdx.x];
  const ByteInfo bi = classify(text, len, p0, x, li0, ls0, fastq);
  if (bi.bad) atomicOr(err, 1u);
  // newline positions: line li ends at its '\n'
  uint64_t li = li0;
#pragma unroll
  for (int i = 0; i < kBpt; ++i)
    if ((bi.nl >> i) & 1u) line_end[li++] = p0 + i;
  uint32_t tk = 0, tr = 0;
  block_excl_sum((uint32_t)__popc(bi.keep), sh, &tk);
  block_excl_sum((uint32_t)__popc(bi.rstart), sh, &tr);
  if (threadIdx.x == 0) {
    tile_keep[blockIdx.x] = tk;
    tile_rec[blockIdx.x] = tr;
  }
}

// (C) per tile: compaction of kept bytes, record offsets.
__global__ void __launch_bounds__(kTpb) pass_c(const uint8_t* __restrict__ text, uint64_t len,
                                                int fastq, const uint64_t* nl_hi,
                                                const int64_t* ls_base, const uint64_t* keep_hi,
                                                const uint64_t* rec_hi, uint8_t* __restrict__ out,
                                                uint64_t* off, uint64_t max_records) {
  __shared__ uint32_t sh[32];
  __shared__ int64_t shm[32];
  const uint64_t p0 = blockIdx.x * kTile + (uint64_t)threadIdx.x * kBpt;
  const Bytes16 x = load_bytes(text, len, p0);
  uint32_t nl = 0;
  int64_t ls = -1;
  uint32_t prev = p0 == 0 ? '\n' : (p0 <= len ? text[p0 - 1] : 0);
#pragma unroll
  for (int i = 0; i < kBpt; ++i) {
    if (p0 + i < len) {
      if (prev == '\n') ls = (int64_t)(p0 + i);
      nl += x.b[i] == '\n';
    }
    prev = x.b[i];
  }
  const uint64_t li0 = nl_hi[blockIdx.x] + block_excl_sum(nl, sh, nullptr);
  int64_t ls0 = block_excl_max(ls, shm);
  if (ls_base[blockIdx.x] > ls0) ls0 = ls_base[blockIdx.x];
  const ByteInfo bi = classify(text, len, p0, x, li0, ls0, fastq);
  uint64_t k = keep_hi[blockIdx.x] + block_excl_sum((uint32_t)__popc(bi.keep), sh, nullptr);
  uint64_t r = rec_hi[blockIdx.x] + block_excl_sum((uint32_t)__popc(bi.rstart), sh, nullptr);
#pragma unroll
  for (int i = 0; i < kBpt; ++i) {
    if ((bi.rstart >> i) & 1u) {
      if (r < max_records) off[r] = k;  // the record's sequence starts after what is kept so far
      ++r;
    }
    if ((bi.keep >> i) & 1u) out[k++] = x.b[i];
  }
}

// FASTQ: record r's quality line (line 4r+3) has as many bytes (without a
// final '\r') as its sequence.
__global__ void check_quality(const uint8_t* __restrict__ text, const uint64_t* line_end,
                              const uint64_t* off, uint64_t n_records, uint32_t* err) {
  for (uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; r < n_records;
       r += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t qs = line_end[4 * r + 2] + 1, qe = line_end[4 * r + 3];
    uint64_t ql = qe - qs;
    if (ql > 0 && text[qe - 1] == '\r') --ql;
    if (ql != off[r + 1] - off[r]) atomicOr(err, 1u);
  }
}

}  // namespace

namespace {

// Scratch layout for a text of `len` bytes (all parts 16-byte aligned).
struct Scratch {
  uint64_t* totals;   // [0] error flag, [1] lines, [2] kept bytes, [3] records
  uint64_t *nl_hi, *keep_hi, *rec_hi;
  int64_t* ls;
  uint32_t *tile_nl, *tile_keep, *tile_rec;
  uint64_t *ga, *gb;
  int64_t* gm;
  uint64_t* line_end;
  uint64_t bytes;
};

inline uint64_t up16(uint64_t x) { return (x + 15) / 16 * 16; }

Scratch layout(uint8_t* base, uint64_t len) {
  const uint64_t tiles = (len + kTile - 1) / kTile + 1;
  const uint64_t groups = (tiles + kScan - 1) / kScan + 1;
  Scratch s{};
  uint64_t at = 0;
  auto take = [&](uint64_t n) {
    uint8_t* p = base ? base + at : nullptr;
    at += up16(n);
    return p;
  };
  s.totals = reinterpret_cast<uint64_t*>(take(64));
  s.nl_hi = reinterpret_cast<uint64_t*>(take(tiles * 8));
  s.keep_hi = reinterpret_cast<uint64_t*>(take(tiles * 8));
  s.rec_hi = reinterpret_cast<uint64_t*>(take(tiles * 8));
  s.ls = reinterpret_cast<int64_t*>(take(tiles * 8));
  s.tile_nl = reinterpret_cast<uint32_t*>(take(tiles * 4));
  s.tile_keep = reinterpret_cast<uint32_t*>(take(tiles * 4));
  s.tile_rec = reinterpret_cast<uint32_t*>(take(tiles * 4));
  s.ga = reinterpret_cast<uint64_t*>(take(groups * 8));
  s.gb = reinterpret_cast<uint64_t*>(take(groups * 8));
  s.gm = reinterpret_cast<int64_t*>(take(groups * 8));
  s.line_end = reinterpret_cast<uint64_t*>(take((len + 1) * 8));
  s.bytes = at;
  return s;
}

}  // namespace

extern "C" {

int sbf_fastx_device_scratch(uint64_t text_len, uint64_t* scratch_bytes) {
  sbf::clear_error();
  if (!scratch_bytes) return fail(SBF_EINVAL, "NULL argument");
  *scratch_bytes = layout(nullptr, text_len).bytes;
  return SBF_OK;
}

int sbf_fastx_parse_device(const uint8_t* d_text, uint64_t text_len, int fastq, uint8_t* d_seq,
                           uint64_t* d_off, uint64_t max_records, void* d_scratch,
                           uint64_t scratch_bytes, uint64_t* h_result, sbf_stream_t stream) {
  sbf::clear_error();
  if (!h_result || (text_len && (!d_text || !d_seq || !d_off || !d_scratch)))
    return fail(SBF_EINVAL, "NULL argument");
  if (reinterpret_cast<uintptr_t>(d_text) % 16 != 0 || reinterpret_cast<uintptr_t>(d_scratch) % 16 != 0)
    return fail(SBF_EINVAL, "d_text and d_scratch must be 16-byte aligned");
  const Scratch sc = layout(static_cast<uint8_t*>(d_scratch), text_len);
  if (scratch_bytes < sc.bytes)
    return fail(SBF_EINVAL, "scratch too small (%llu < %llu bytes)", (unsigned long long)scratch_bytes,
                (unsigned long long)sc.bytes);
  h_result[0] = h_result[1] = h_result[2] = 0;
  if (text_len == 0) return SBF_OK;
  if (text_len >= (1ull << 40)) return fail(SBF_EINVAL, "text too long");
  cudaStream_t st = (cudaStream_t)stream;
  const uint64_t tiles = (text_len + kTile - 1) / kTile;
  uint32_t* err = reinterpret_cast<uint32_t*>(sc.totals);
  cudaError_t e;
  if ((e = cudaMemsetAsync(sc.totals, 0, 64, st)) != cudaSuccess) return cuda_fail(e, "fastx scratch");
  pass_a<<<(int)tiles, kTpb, 0, st>>>(d_text, text_len, sc.tile_nl, sc.ls);
  ScanIO s1{sc.tile_nl, nullptr, sc.ls, sc.nl_hi, nullptr, sc.ls, sc.ga, sc.gb, sc.gm, tiles,
            sc.totals + 1};
  if ((e = scan3(s1, st)) != cudaSuccess) return cuda_fail(e, "fastx scan");
  pass_b<<<(int)tiles, kTpb, 0, st>>>(d_text, text_len, fastq, sc.nl_hi, sc.ls, sc.tile_keep,
                                       sc.tile_rec, sc.line_end, err);
  ScanIO s2{sc.tile_keep, sc.tile_rec, nullptr, sc.keep_hi, sc.rec_hi, nullptr, sc.ga, sc.gb, sc.gm,
            tiles, sc.totals + 2};
  if ((e = scan3(s2, st)) != cudaSuccess) return cuda_fail(e, "fastx scan");
  uint64_t tot[4];
  if ((e = cudaMemcpyAsync(tot, sc.totals, sizeof(tot), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
      (e = cudaStreamSynchronize(st)) != cudaSuccess)
    return cuda_fail(e, "fastx totals");
  const uint64_t n_lines = tot[1], kept = tot[2], n_rec = tot[3];
  bool bad = (tot[0] & 0xFFFFFFFFull) != 0;
  if (fastq && n_lines != 4 * n_rec) bad = true;
  if (!bad && n_rec > max_records)
    return fail(SBF_EINVAL, "%llu records exceed max_records", (unsigned long long)n_rec);
  if (!bad) {
    pass_c<<<(int)tiles, kTpb, 0, st>>>(d_text, text_len, fastq, sc.nl_hi, sc.ls, sc.keep_hi,
                                         sc.rec_hi, d_seq, d_off, max_records);
    if ((e = cudaMemcpyAsync(d_off + n_rec, &sc.totals[2], 8, cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
      return cuda_fail(e, "fastx offsets");
    if (fastq && n_rec) {
      const uint64_t blocks = (n_rec + 255) / 256;
      check_quality<<<(int)(blocks < 4096 ? blocks : 4096), 256, 0, st>>>(d_text, sc.line_end, d_off,
                                                                         n_rec, err);
    }
    uint64_t e2 = 0;
    if ((e = cudaMemcpyAsync(&e2, sc.totals, 8, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
      return cuda_fail(e, "fastx compaction");
    bad = (e2 & 0xFFFFFFFFull) != 0;
  }
  h_result[0] = n_rec;
  h_result[1] = kept;
  h_result[2] = bad ? 1 : 0;
  return SBF_OK;
}

}  // extern "C"
