// msa_kernels.cuh -- encode, traceback, merge, rows, SP and center kernels.
#pragma once
#include "common.cuh"

cudaError_t launch_encode(const uint8_t *letters, const int64_t *src_off, const int32_t *perm,
                          const int64_t *pstart, const int32_t *len, int n, const uint8_t *lut,
                          int padc, uint8_t *res, unsigned *err, cudaStream_t st);

// res/pstart/center/M/K/o/e: the walk recomputes the score of each cell on
// its path (the codes hold a source only where H > 0).
// list: subjects by sorted index (else [sb, se)), their best cells then read
// at best[k]; box (with list): per list position {first row, rows, first
// column, columns} of the box its codes cover, box_best the box's own best
// cell (it must be the matrix's best cell in box coordinates).
cudaError_t launch_traceback(const uint8_t *codes, const int64_t *code_off,
                             const unsigned long long *best,
                             int sb, int se, const int32_t *len, const int32_t *perm,
                             const uint8_t *res, const int64_t *pstart, int center,
                             const int8_t *M, int K, int o, int e, int Lc, int G,
                             uint16_t *ins, uint8_t *occ, int32_t *seg, int32_t *score,
                             unsigned *err, cudaStream_t st, const int32_t *list = nullptr,
                             const int4 *box = nullptr,
                             const unsigned long long *box_best = nullptr);

cudaError_t launch_colmax(const uint16_t *ins, int n, int Lc, int32_t *G, cudaStream_t st);
cudaError_t launch_scan(const int32_t *G, int Lc, int32_t *off, int64_t *width, cudaStream_t st);
cudaError_t launch_rows(const uint8_t *res, const int64_t *pstart, const int32_t *inv,
                        const uint16_t *ins, const uint8_t *occ, const int32_t *G,
                        const int32_t *off, int n, int Lc, int64_t W, const char *letters,
                        uint8_t *out, cudaStream_t st);
cudaError_t launch_sp(const uint8_t *msa, int n, int64_t W, const uint8_t *sym_lut, int nsym,
                      int32_t *counts, unsigned long long *total, cudaStream_t st);

// Row sums of the center distance from the similarity sums (mode 0: all
// pairs, mode 1: nref references) and their argmin (lowest input index).
cudaError_t launch_center_finalize(int mode, int n, int nref, const int32_t *perm,
                                   const unsigned long long *pairsum, long long *rowsum,
                                   long long *argmin_val, long long *argmin_idx,
                                   long long *part_val, long long *part_idx, cudaStream_t st);

cudaError_t launch_apply_overflow(int mode, const int2 *ovf, const int32_t *scores, int count,
                                  unsigned long long *pairsum, const int32_t *self, cudaStream_t st);

cudaError_t launch_self_pairs(int n, int2 *pairs, int32_t *dst, cudaStream_t st);
cudaError_t launch_extract_scores(const int32_t *seg, int n, int32_t *out, cudaStream_t st);
