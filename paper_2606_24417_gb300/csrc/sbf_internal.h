// sbf_internal.h -- host-side internals of libsbf shared by the C ABI and the
// kernel launchers.
#pragma once

#include <cstdint>
#include <mutex>

#include <cuda_runtime.h>

#include "sbf.h"
#include "sbf_device.cuh"

struct sbf_filter {
  sbf::Geom geom;
  int device = 0;
  uint64_t n_words = 0;
  bool fused = false;  // a specialised kernel exists for these parameters
  // kernels that serve the filter: 1 fused, 2 rolling (every other parameter
  // set), 0 generic one-k-mer-per-thread (only when SBF_FORCE_GENERIC is set)
  int variant = 0;
  // host-input path (sbf_*_host): reusable device buffers and two streams
  std::mutex host_mu;
  cudaStream_t host_streams[2] = {nullptr, nullptr};
  uint8_t* host_dev_seq[2] = {nullptr, nullptr};
  uint64_t* host_dev_off[2] = {nullptr, nullptr};
  uint32_t* host_dev_bits[2] = {nullptr, nullptr};
  uint32_t* host_dev_hits[2] = {nullptr, nullptr};
  uint64_t host_cap_seq = 0, host_cap_reads = 0;
  // pinned landing slots for each chunk's first answer word (a pageable
  // destination would make the copy synchronous and stall the pipeline)
  uint32_t* host_first = nullptr;
  uint64_t host_first_cap = 0;
  // pinned staging of a chunk's answers when the caller's output buffers are
  // pageable (a copy into pageable memory would wait for the chunk's kernel
  // and stop the next chunk's upload from overlapping it)
  uint32_t* host_stage_bits[2] = {nullptr, nullptr};
  uint32_t* host_stage_hits[2] = {nullptr, nullptr};
  uint64_t host_stage_words = 0, host_stage_reads = 0;
};

namespace sbf {

// Thread-local error message; returns `code` for convenient `return fail(...)`.
int fail(int code, const char* fmt, ...);
int cuda_fail(cudaError_t e, const char* what);
void clear_error();

// Generic kernels: any valid parameter set, one k-mer per thread.
cudaError_t generic_insert(const Geom& g, const uint8_t* seq, uint64_t seq_len,
                           const uint64_t* off, uint64_t n_reads, cudaStream_t st);
cudaError_t generic_query(const Geom& g, const uint8_t* seq, uint64_t seq_len,
                          const uint64_t* off, uint64_t n_reads, uint32_t* bits, uint32_t* hits,
                          uint64_t* stats, cudaStream_t st);

// Rolling kernels: any valid parameter set, one thread per 32 start positions.
cudaError_t rolling_insert(const Geom& g, const uint8_t* seq, uint64_t seq_len,
                           const uint64_t* off, uint64_t n_reads, cudaStream_t st);
cudaError_t rolling_query(const Geom& g, const uint8_t* seq, uint64_t seq_len,
                          const uint64_t* off, uint64_t n_reads, uint32_t* bits, uint32_t* hits,
                          uint64_t* stats, cudaStream_t st);

// Fused kernels: the compiled (w, H, B) grid.
bool fused_supported(const Geom& g);
cudaError_t fused_insert(const Geom& g, const uint8_t* seq, uint64_t seq_len, const uint64_t* off,
                         uint64_t n_reads, cudaStream_t st);
cudaError_t fused_query(const Geom& g, const uint8_t* seq, uint64_t seq_len, const uint64_t* off,
                        uint64_t n_reads, uint32_t* bits, uint32_t* hits, uint64_t* stats,
                        cudaStream_t st);

// Number of SMs of the current device (cached).
int sm_count();

}  // namespace sbf
