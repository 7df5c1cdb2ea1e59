// sw_kernels.cuh -- launch interfaces of the Smith-Waterman kernels.
#pragma once
#include "common.cuh"

// Per-sequence device layout produced by the encode kernel (sorted order).
struct SeqSet {
  const uint8_t *res;     // residues (alphabet index; padding code = K), 16-B aligned per sequence
  const int64_t *pstart;  // start of sequence k in res
  const int32_t *len;     // length of sequence k
  int n;
};

struct Scoring {
  const int8_t *M;        // K x K, device
  int K, o, e;
};

// All-pairs / reference-pairs scores for center selection.
struct CenterJob {
  int mode;                       // 0: query q vs subjects (q, n), both sides summed;
                                  // 1: query qlist[x] vs [0, n), summed on the subject;
                                  // 2: query qlist[x] vs [0, n), summed on the query
  const int32_t *qlist;           // mode 1 (sorted indices)
  int nq;                         // queries in the list (mode 0: n)
  int qb, qe;                     // item-unit range: queries (single) or query pairs (paired)
  int sub_off, sub_n;             // modes 1, 2: subjects [sub_off, sub_off + sub_n)
  const int64_t *prefix;          // device, qe-qb+1 entries: first item of each query
  int64_t n_items;
  int npass;                      // passes of the longest query in the range
  unsigned long long *counter;    // zeroed before launch
  unsigned long long *pairsum;    // sums of center_sim over the listed partners (job's index)
  const int32_t *self;            // S(k,k) of every sequence in the job's index space (read)
  int sat_thresh;                 // packed cells: lanes whose best exceeds this are re-run in int32
  int2 *ovf; unsigned *ovf_count; int ovf_cap; unsigned *err;
  int2 *scratch; int scratch_cols;
  // paired classes: the unit is a stream of consecutive query pairs stacked
  // in one row range, streams[u] = {first pair, pair count <= kMaxSeg}
  const int2 *streams;
};

// Query pairs one stream of the paired center kernel may stack.
constexpr int kMaxSeg = 32;

// Arbitrary pair list (int32 cells).
struct PairJob {
  const int2 *pairs;              // (a, b) sorted indices; a = rows (query), b = columns
  const int32_t *dst;             // output slot of each listed pair
  int32_t *out;
  int npairs;
  unsigned long long *counter;
  int2 *scratch; int scratch_cols;
};

// Alignment to the center with 4-bit traceback codes (int32 cells, or two
// subjects per group in the int16 lanes when packed).
struct CodesJob {
  int center;                     // sorted index
  int sb, se;                     // subjects: sorted indices [sb, se), longest first
  const int64_t *code_off;        // byte offset of each subject's codes (indexed k - sb)
  uint8_t *codes;
  unsigned long long *best;       // per subject (indexed k - sb): best_key of its best cell
  int npass;
  unsigned long long *counter;
  int2 *scratch; int scratch_cols;
};

// Kernel variants of center selection: paired = two queries in the int16
// lanes (k_center2), else one query with two packed subjects or int32 cells.
struct CenterVariant { int paired, G, R; bool packed; };
extern const CenterVariant kCenterVariants[];
extern const int kNumCenterVariants;

// dynamic shared memory of a center launch whose units need rows_alloc
// profile rows; center_profile_bytes: the profile part alone
int center_smem_bytes(int variant, int K, int rows_alloc);
int center_profile_bytes(int variant, int K, int rows_alloc);
// set_smem = false: the caller has already raised the kernel's dynamic
// shared-memory limit with center_allow_smem (required while a stream is
// being captured into a graph).
cudaError_t launch_center(int variant, const SeqSet &ss, const Scoring &sc, const CenterJob &job,
                          int grid, cudaStream_t st, bool set_smem = true);
cudaError_t center_allow_smem(int variant, int smem);
int center_grid(int variant, int smem);

cudaError_t launch_pairs(int G, const SeqSet &ss, const Scoring &sc, const PairJob &job,
                         int grid, cudaStream_t st);
int pairs_grid(int G);
int pairs_rows(int G);

// G = threads per subject group (1, 2, 4, 8, 16 or 32; codes_group picks 8-32 from the
// center length and the subject lengths); 16 center rows per thread.  packed: each group carries two
// subjects in int16 lanes (the caller checks that every cell value fits).
// set_smem = false: the caller has already raised the kernel's dynamic
// shared-memory limit with codes_allow_smem (required while capturing).
// threads: CTA size of the packed kernel (kCodes2Threads or, for G >= 8,
// kCodes2WideThreads); the int32 kernel always runs kCodes2Threads.
cudaError_t launch_codes(int G, bool packed, const SeqSet &ss, const Scoring &sc, const CodesJob &job,
                         int grid, cudaStream_t st, bool set_smem = true, int threads = 256);
cudaError_t codes_allow_smem(int G, bool packed, int smem, int threads = 256);
int codes_smem_bytes(int K, int rows_alloc);
int codes_grid(int G, bool packed, int smem, int threads = 256);
int codes_threads(bool packed, int threads = 256);  // threads per CTA of the codes kernels
int codes_group(int Lc, bool packed, int K, int64_t n, double mean_len, int max_len);
constexpr int kCodesR = 16;
// lanes per subject the alignment kernels come in: 1, 2, 4, 8, 16, 32
constexpr int kAlignWidths = 6;
constexpr int kCodes2Threads = 256;      // codes kernel threads per CTA
constexpr int kCodes2WideThreads = 384;  // the packed kernel's wider CTA
constexpr int kPairsR = 16;
constexpr int kCenterThreads = 256;

// The traceback-light alignment to the center, packed cells only: a forward
// score pass to each subject's best cell (mode 1), a pass over the reversed
// prefixes up to that cell to where best-scoring alignments may start
// (mode 2), and the codes of the box between (mode 3).
struct LightJob {
  int center;                     // sorted index
  int sb, se, npass;              // mode 1: subjects [sb, se) in sorted order, passes over the center
  int npos;                       // modes 2, 3: positions; group x takes positions 2x and 2x+1
  const int32_t *order;           // modes 2, 3: sorted subject index of each position
  const int4 *win;                // modes 2, 3: per position {first profile row (a multiple of
                                  // 16), rows, mode 2: masked top rows / mode 3: first column,
                                  // columns}
  const int64_t *code_off;        // mode 3: byte offset of each position's codes
  uint8_t *codes;
  unsigned long long *best;       // mode 1: per subject (k - sb); modes 2, 3: per position
  unsigned long long *counter;
  int2 *scratch; int scratch_cols;
};
// profile rows of a light pass (modes 2 and 3 hold the whole center, and the
// center reversed for mode 2, plus two passes of padding rows)
__host__ __device__ inline int light_prof_rows(int Lc, int G, int mode, int npass) {
  return mode == 1 ? npass * G * 16 : ((Lc + 15) & ~15) + 2 * G * 16;
}
int light_smem_bytes(int K, int Lc, int G, int mode, int npass);
cudaError_t light_allow_smem(int G, int mode, int smem);
int light_grid(int G, int mode, int smem);
cudaError_t launch_light(int G, int mode, const SeqSet &ss, const Scoring &sc, const LightJob &job,
                         int grid, int smem, cudaStream_t st);
constexpr int kLightThreads = 256;
