// cg_launch.h -- host-side launch wrappers of libcg's kernels.  All
// return the cudaError_t of the launch.
#pragma once
#include "cg_internal.h"

namespace cgi {

// Launch wrappers (cg_kernels.cu).  All return cudaError_t of the launch.
cudaError_t launch_init_single_scratch(SingleScratch *s, cudaStream_t st);
cudaError_t launch_scan_single(const Image &img, const ScanJob &job, const RangeInfo &ri,
                               SingleScratch *scratch, cg_report *out, int grid,
                               cudaStream_t st);
int scan_single_max_ctas_per_sm(uint32_t kind, uint32_t mode);
cudaError_t launch_scan_single_tma(const Image &img, const ScanJob &job, const RangeInfo &ri,
                                   SingleScratch *scr, cg_report *out, int grid,
                                   cudaStream_t st);
int scan_single_tma_grid(int sm_count, uint64_t n);
uint32_t scan_tma_tile_bytes();  // a batched segment is a whole number of these
// The reports of a one-level plan written by the level kernel's last CTA
// straight into pinned host memory (out: error flag (16 bytes) | reports;
// done: a zeroed CTA counter), or nothing (out null).
struct FinalizeHost {
  uint8_t *out = nullptr;
  unsigned int *done = nullptr;
};

// claim: per-level counter, zero before the launch (dynamic segment
// claiming), or null (static striding).  overlap: launched as a
// programmatic dependent of the kernel before it on `st` (its prologue
// overlaps that kernel's tail; it waits for it before reading shadow).
cudaError_t launch_scan_level_tma(const Image &img, const BatchPlan &p, uint64_t pos_begin,
                                  uint64_t pos_end, uint64_t n_segs, int max_ctas,
                                  unsigned long long *claim, unsigned int *err_flag, bool overlap,
                                  cudaStream_t st, const FinalizeHost &fin = FinalizeHost{});
// New device table = old minus the entries whose bases are in the sorted
// list `dead`, plus the sorted registrations, into nb/ns/nh (count - d + m
// entries).
cudaError_t launch_table_merge(const DevTable &t, const uint64_t *ins_base,
                               const uint64_t *ins_size, const uint64_t *ins_shadow, uint64_t m,
                               const uint64_t *dead, uint64_t d, uint64_t *nb, uint64_t *ns,
                               uint64_t *nh, int sm_count, cudaStream_t st);
cudaError_t launch_lookup(const DevTable &t, const BatchPlan &p, int strict, int carry,
                          cudaStream_t st);
cudaError_t launch_job_modes(const BatchPlan &p, uint8_t *modes, cudaStream_t st);
cudaError_t launch_scan_level(const Image &img, const BatchPlan &p, uint64_t pos_begin,
                              uint64_t pos_end, uint64_t n_segs, int grid, cudaStream_t st);
// The error flag and the reports into `out` (pinned host memory the
// kernel writes directly): flag (16 bytes) | nreq reports.
cudaError_t launch_finalize_host(const BatchPlan &p, const unsigned int *err, uint8_t *out,
                                  cudaStream_t st);
cudaError_t launch_finalize(const BatchPlan &p, cg_report *reps, uint32_t *counts,
                            uint64_t *block_sums, int items_per_block, cudaStream_t st);
cudaError_t launch_scan_block_sums(uint64_t *block_sums, uint64_t nblocks, uint64_t *total,
                                   cudaStream_t st);
cudaError_t launch_emit_records(const BatchPlan &p, const cg_report *reps, const uint32_t *counts,
                                const uint64_t *block_sums, int items_per_block, int strict,
                                cg_err_record *recs, uint64_t rec_cap, cudaStream_t st);
cudaError_t launch_fill(const uint64_t *ptrs, const uint64_t *sizes, uint64_t count,
                        uint8_t value, cudaStream_t st);

// Pitched copies (cg_scan_pitched.cu).
// row_chunks = 16-byte chunks of the longest row on its anchor grid;
// tma_ok = bulk copies may read the image (it is in device memory).
cudaError_t launch_scan_pitched(const Image &img, const PitchedJob &job, const RangeInfo &ri,
                                SingleScratch *scr, cg_report *out, int sm_count,
                                uint64_t row_chunks, bool tma_ok, cudaStream_t st);
// Gather the rows of a pitched device span into dense `out` (row-major).
cudaError_t launch_gather_rows(const uint8_t *src, uint64_t pitch, uint64_t slice,
                               uint64_t width, uint64_t height, uint64_t depth, uint8_t *out,
                               int sm_count, cudaStream_t st);

// Memset and kernel arguments (cg_devops_kernels.cu).
cudaError_t launch_fill_rows(uint8_t *base, uint64_t pitch, uint64_t width, uint64_t rows,
                             uint8_t value, const RangeInfo &ri, cg_report *out, int sm_count,
                             cudaStream_t st);
uint64_t fill_span_groups(uint64_t n);  // fill groups of a span of n bytes
cudaError_t launch_fill_spans(const uint64_t *ptr, const uint64_t *n, const uint64_t *seg_first,
                              uint64_t count, uint64_t nsegs, uint8_t value, int sm_count,
                              cudaStream_t st);

}  // namespace cgi
