/*
 * msa_oracle.c -- plain, slow CPU oracle for the center-star MSA hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code, header,
 * table or helper with the CUDA path; it is written from the paper
 * (HAlign-II, arXiv 1704.00878) and the readings listed below.
 *
 * Every routine is the plain definition: full (Lc+1) x (Ls+1) matrices,
 * scalar loops, no blocking, tiling or vectorisation.  Threads are used only
 * across independent pairs (one pair = one task).
 *
 * Conventions shared with the callers (inputs only):
 *   residues are alphabet indices 0..K-1; M is a K x K int8 matrix, row-major,
 *   s(a, b) = M[a*K + b]; the center c indexes rows i = 1..Lc and the other
 *   sequence s indexes columns j = 1..Ls.
 *
 * Readings of the paper taken here (the paper is silent or ambiguous):
 *   - gap weight W_k = o + (k-1)e with o >= e > 0, the same for both gap
 *     directions (Eq. 2 writes W_k and W_l);
 *   - best cell: the maximum H with the smallest i, then the smallest j;
 *   - traceback ties (H > 0): diagonal, then vertical gap (F), then horizontal
 *     gap (E); a gap extends only when extending is strictly better than
 *     opening;
 *   - residues outside the local segment: prefix right-aligned and suffix
 *     left-aligned without gaps; excess sequence residues go to insertion slot 0
 *     (prefix) or slot Lc (suffix), excess center residues face a gap;
 *   - inserted residues are left-justified in their slot, gaps follow;
 *   - center (Figure 3: "extracted ... based on Smith-Waterman"; the trie
 *     paragraph: the sequence "most similar to other sequences"): similarity of
 *     a pair = its local score as a fraction of the larger self score,
 *     S(A,B) / max(S(A,A), S(B,B)), held in 16-bit fixed point; distance
 *     d(A,B) = 2^16 - floor(2^16 S(A,B) / max(S(A,A), S(B,B))), and d = 0 when
 *     both self scores are 0; center = argmin of the row sums of d, lowest
 *     index on ties.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>
#include <stdatomic.h>
#include <unistd.h>

#define ORC_NEG (-(1 << 29)) /* stands for minus infinity in E and F */

static int32_t max2(int32_t a, int32_t b) { return a > b ? a : b; }

/*
 * Smith-Waterman local alignment with affine gaps, Eq. (1)-(2): the general
 * gap terms max_k {H[i-k][j] - W_k} and max_l {H[i][j-l] - W_l} are carried by
 * Gotoh's two auxiliary matrices, which equal them exactly for
 * W_k = o + (k-1)e:
 *   E[i][j] = max(H[i][j-1] - o, E[i][j-1] - e)       (gap in the center)
 *   F[i][j] = max(H[i-1][j] - o, F[i-1][j] - e)       (gap in the sequence)
 *   H[i][j] = max(0, H[i-1][j-1] + s(c_i, s_j), E[i][j], F[i][j])
 * with H[0][*] = H[*][0] = 0 (Eq. 1) and E[*][0] = F[0][*] = -inf.
 *
 * codes (nullable): Lc*Ls bytes, codes[(i-1)*Ls + (j-1)] =
 *     src | (E extended) << 2 | (F extended) << 3,
 *   src = 0 if H == 0, 1 if H came from the diagonal, 2 from F, 3 from E.
 * end (nullable): end[0] = i, end[1] = j of the best cell (0, 0 if best == 0).
 * Returns max H (>= 0), or -1 if out of memory.
 */
int32_t orc_sw(const uint8_t *c, int32_t lc, const uint8_t *s, int32_t ls,
               const int8_t *M, int32_t K, int32_t o, int32_t e,
               uint8_t *codes, int32_t *end)
{
    size_t w = (size_t)ls + 1;
    size_t cells = ((size_t)lc + 1) * w;
    int32_t *H = malloc(cells * sizeof(int32_t));
    int32_t *E = malloc(cells * sizeof(int32_t));
    int32_t *F = malloc(cells * sizeof(int32_t));
    if (!H || !E || !F) { free(H); free(E); free(F); return -1; }

    for (size_t j = 0; j < w; j++) { H[j] = 0; E[j] = ORC_NEG; F[j] = ORC_NEG; }
    for (int32_t i = 1; i <= lc; i++) {
        H[i * w] = 0; E[i * w] = ORC_NEG; F[i * w] = ORC_NEG;
    }

    int32_t best = 0, bi = 0, bj = 0;
    for (int32_t i = 1; i <= lc; i++) {
        for (int32_t j = 1; j <= ls; j++) {
            size_t at = (size_t)i * w + j;
            int32_t e_open = H[at - 1] - o, e_ext = E[at - 1] - e;
            int32_t f_open = H[at - w] - o, f_ext = F[at - w] - e;
            int32_t ev = max2(e_open, e_ext);
            int32_t fv = max2(f_open, f_ext);
            int32_t dv = H[at - w - 1] + M[c[i - 1] * K + s[j - 1]];
            int32_t hv = max2(max2(0, dv), max2(ev, fv));
            E[at] = ev; F[at] = fv; H[at] = hv;
            if (codes) {
                int32_t src = hv == 0 ? 0 : (hv == dv ? 1 : (hv == fv ? 2 : 3));
                codes[(size_t)(i - 1) * ls + (j - 1)] =
                    (uint8_t)(src | ((e_ext > e_open) << 2) | ((f_ext > f_open) << 3));
            }
            if (hv > best) { best = hv; bi = i; bj = j; }
        }
    }
    if (end) { end[0] = bi; end[1] = bj; }
    free(H); free(E); free(F);
    return best;
}

/*
 * Traceback (the paper: from the highest-scoring cell back to a cell whose
 * score is zero) followed by the flank rule, producing the row's entry in the
 * inserted-space matrix:
 *   ins[j], j = 0..Lc: sequence residues placed between c_j and c_{j+1}
 *                      (slot 0 before c_1, slot Lc after c_Lc);
 *   occ[i], i = 1..Lc: 1 if a sequence residue faces c_i, 0 if a gap does
 *                      (occ[0] is unused and set to 0).
 * seg (nullable) = {i1, j1, i2, j2}: the local segment is
 * c[i1+1..i2] x s[j1+1..j2]; all zero when best == 0.
 * Returns 0, or -1 if the codes are inconsistent.
 */
int orc_traceback(const uint8_t *codes, int32_t lc, int32_t ls, int32_t best,
                  int32_t i2, int32_t j2, uint16_t *ins, uint8_t *occ, int32_t *seg)
{
    memset(ins, 0, sizeof(uint16_t) * ((size_t)lc + 1));
    memset(occ, 0, (size_t)lc + 1);
    int32_t i1 = 0, j1 = 0;
    if (best == 0) { i2 = 0; j2 = 0; }
    else {
        int32_t i = i2, j = j2;
        int state = 0; /* 0 = H, 1 = F (vertical gap), 2 = E (horizontal gap) */
        for (;;) {
            if (i <= 0 || j <= 0) {
                if (state != 0) return -1;
                break; /* H is zero on row 0 and column 0 */
            }
            uint8_t code = codes[(size_t)(i - 1) * ls + (j - 1)];
            if (state == 0) {
                int src = code & 3;
                if (src == 0) break;
                if (src == 1) { occ[i] = 1; i--; j--; }
                else if (src == 2) state = 1;
                else state = 2;
            } else if (state == 1) {           /* c_i faces a gap */
                state = (code >> 3) & 1 ? 1 : 0;
                i--;
            } else {                           /* s_j inserted after c_i */
                ins[i]++;
                state = (code >> 2) & 1 ? 2 : 0;
                j--;
            }
        }
        i1 = i; j1 = j;
    }
    /* prefix: right-aligned, no gaps */
    int32_t k = i1 < j1 ? i1 : j1;
    for (int32_t t = 0; t < k; t++) occ[i1 - t] = 1;
    if (j1 > i1) ins[0] += (uint16_t)(j1 - i1);
    /* suffix: left-aligned, no gaps */
    int32_t a = lc - i2, b = ls - j2;
    k = a < b ? a : b;
    for (int32_t t = 1; t <= k; t++) occ[i2 + t] = 1;
    if (b > a) ins[lc] += (uint16_t)(b - a);
    if (seg) { seg[0] = i1; seg[1] = j1; seg[2] = i2; seg[3] = j2; }
    return 0;
}

/* ---------------------------------------------------------------------- */
/* a minimal thread pool: tasks 0..n-1 pulled from an atomic counter       */

typedef void (*orc_task_fn)(void *ctx, int64_t t);
typedef struct { atomic_llong next; int64_t n; orc_task_fn fn; void *ctx; } orc_pool;

static void *orc_worker(void *arg)
{
    orc_pool *p = arg;
    for (;;) {
        int64_t t = atomic_fetch_add(&p->next, 1);
        if (t >= p->n) break;
        p->fn(p->ctx, t);
    }
    return NULL;
}

int orc_default_threads(void)
{
    long n = sysconf(_SC_NPROCESSORS_ONLN);
    return n > 0 ? (int)n : 1;
}

static void orc_parallel_for(int64_t n, int threads, orc_task_fn fn, void *ctx)
{
    if (threads <= 0) threads = orc_default_threads();
    if (threads > 256) threads = 256;
    orc_pool p; atomic_init(&p.next, 0); p.n = n; p.fn = fn; p.ctx = ctx;
    pthread_t tid[256];
    int started = 0;
    for (int t = 1; t < threads; t++)
        if (pthread_create(&tid[started], NULL, orc_worker, &p) == 0) started++;
    orc_worker(&p);
    for (int t = 0; t < started; t++) pthread_join(tid[t], NULL);
}

/* ---------------------------------------------------------------------- */

typedef struct {
    const uint8_t *res; const int64_t *off;
    const int8_t *M; int32_t K, o, e;
} orc_seqs;

typedef struct { orc_seqs q; const int64_t *pairs; int32_t *out; atomic_int err; } pair_job;

static void pair_task(void *ctx, int64_t t)
{
    pair_job *j = ctx;
    int64_t a = j->pairs[2 * t], b = j->pairs[2 * t + 1];
    const orc_seqs *q = &j->q;
    int32_t v = orc_sw(q->res + q->off[a], (int32_t)(q->off[a + 1] - q->off[a]),
                       q->res + q->off[b], (int32_t)(q->off[b + 1] - q->off[b]),
                       q->M, q->K, q->o, q->e, NULL, NULL);
    if (v < 0) atomic_store(&j->err, 1);
    j->out[t] = v;
}

/* S(a_t, b_t) for every listed pair (a as center/rows, b as columns). */
int orc_pair_scores(const uint8_t *res, const int64_t *off, const int64_t *pairs,
                    int64_t npairs, const int8_t *M, int32_t K, int32_t o, int32_t e,
                    int32_t *out, int threads)
{
    pair_job j = { { res, off, M, K, o, e }, pairs, out, 0 };
    orc_parallel_for(npairs, threads, pair_task, &j);
    return atomic_load(&j.err) ? -1 : 0;
}

typedef struct {
    orc_seqs q; int64_t center; int32_t lc;
    uint16_t *ins; uint8_t *occ; int32_t *seg; atomic_int err;
} align_job;

static void align_task(void *ctx, int64_t t)
{
    align_job *j = ctx;
    const orc_seqs *q = &j->q;
    const uint8_t *c = q->res + q->off[j->center];
    const uint8_t *s = q->res + q->off[t];
    int32_t lc = j->lc, ls = (int32_t)(q->off[t + 1] - q->off[t]);
    uint8_t *codes = malloc((size_t)lc * ls + 1);
    int32_t end[2];
    if (!codes) { atomic_store(&j->err, 1); return; }
    int32_t best = orc_sw(c, lc, s, ls, q->M, q->K, q->o, q->e, codes, end);
    int32_t *seg = j->seg + 5 * t;
    if (best < 0 || orc_traceback(codes, lc, ls, best, end[0], end[1],
                                  j->ins + (size_t)t * (lc + 1),
                                  j->occ + (size_t)t * (lc + 1), seg + 1) != 0)
        atomic_store(&j->err, 1);
    seg[0] = best;
    free(codes);
}

/*
 * Align every sequence to the center (the map step of Figure 3): for row t,
 * seg[5t..5t+4] = {score, i1, j1, i2, j2}, ins[t*(Lc+1) ..] and
 * occ[t*(Lc+1) ..] as in orc_traceback.
 */
int orc_align_all(const uint8_t *res, const int64_t *off, int64_t n, int64_t center,
                  const int8_t *M, int32_t K, int32_t o, int32_t e,
                  uint16_t *ins, uint8_t *occ, int32_t *seg, int threads)
{
    align_job j = { { res, off, M, K, o, e }, center,
                    (int32_t)(off[center + 1] - off[center]), ins, occ, seg, 0 };
    orc_parallel_for(n, threads, align_task, &j);
    return atomic_load(&j.err) ? -1 : 0;
}

/*
 * The reduce step of Figure 3: the inserted-space matrix ins (n x (Lc+1))
 * gives, per slot, the largest number of residues any row inserts there:
 * G[j] = max_t ins[t][j].  Returns the MSA width W = Lc + sum_j G[j].
 */
int64_t orc_merge_width(const uint16_t *ins, int64_t n, int32_t lc, int32_t *G)
{
    int64_t w = lc;
    for (int32_t j = 0; j <= lc; j++) {
        int32_t g = 0;
        for (int64_t t = 0; t < n; t++) {
            int32_t v = ins[(size_t)t * (lc + 1) + j];
            if (v > g) g = v;
        }
        G[j] = g;
        w += g;
    }
    return w;
}

/*
 * The final map step of Figure 3: every row re-expanded against the merged
 * ("longest") center.  Slot j holds the row's ins[j] inserted residues, then
 * G[j] - ins[j] gaps; center column j+1 holds the facing residue or a gap.
 * letters[k] is the character of alphabet index k.  out is n x W bytes.
 */
int orc_write_rows(const uint8_t *res, const int64_t *off, int64_t n, int32_t lc,
                   const uint16_t *ins, const uint8_t *occ, const int32_t *G,
                   int64_t width, const char *letters, uint8_t *out)
{
    for (int64_t t = 0; t < n; t++) {
        const uint8_t *s = res + off[t];
        int64_t ls = off[t + 1] - off[t], k = 0, pos = 0;
        const uint16_t *in = ins + (size_t)t * (lc + 1);
        const uint8_t *oc = occ + (size_t)t * (lc + 1);
        uint8_t *row = out + (size_t)t * width;
        for (int32_t j = 0; j <= lc; j++) {
            for (int32_t u = 0; u < in[j]; u++) row[pos++] = (uint8_t)letters[s[k++]];
            for (int32_t u = in[j]; u < G[j]; u++) row[pos++] = '-';
            if (j < lc) row[pos++] = oc[j + 1] ? (uint8_t)letters[s[k++]] : '-';
        }
        if (pos != width || k != ls) return -1;
    }
    return 0;
}

/*
 * Sum-of-pairs cost as the paper defines it for avg SP: over every pair of
 * rows and every column, +1 for two different residues, +2 for a residue
 * facing a gap, 0 for equal residues or two gaps.  Literal O(n^2 W) loop.
 */
int64_t orc_sp_pairwise(const uint8_t *msa, int64_t n, int64_t width)
{
    int64_t total = 0;
    for (int64_t a = 0; a < n; a++)
        for (int64_t b = a + 1; b < n; b++) {
            const uint8_t *ra = msa + (size_t)a * width, *rb = msa + (size_t)b * width;
            for (int64_t x = 0; x < width; x++) {
                int ga = ra[x] == '-', gb = rb[x] == '-';
                if (ga && gb) continue;
                if (ga || gb) total += 2;
                else if (ra[x] != rb[x]) total += 1;
            }
        }
    return total;
}

/*
 * The same cost counted per column: with R residues, g gaps and count c_a of
 * each residue, differing residue pairs number (R^2 - sum c_a^2)/2 and
 * residue-gap pairs number g*R.
 */
int64_t orc_sp_columns(const uint8_t *msa, int64_t n, int64_t width)
{
    int64_t total = 0;
    int64_t cnt[256];
    for (int64_t x = 0; x < width; x++) {
        memset(cnt, 0, sizeof cnt);
        for (int64_t t = 0; t < n; t++) cnt[msa[(size_t)t * width + x]]++;
        int64_t g = cnt['-'], r = n - g, sq = 0;
        for (int v = 0; v < 256; v++) if (v != '-') sq += cnt[v] * cnt[v];
        total += (r * r - sq) / 2 + 2 * g * r;
    }
    return total;
}

/*
 * Distance of a pair for the exact center, in units of 2^-16:
 *   d(A,B) = 2^16 - floor(2^16 * S(A,B) / m),  m = max(S(A,A), S(B,B)),
 * i.e. one minus the fraction of the larger self score that the pair's local
 * alignment reaches (0 for identical sequences, 2^16 for a pair with no
 * positive local alignment).  d = 0 when m == 0.  S(A,B) >= 0, so the integer
 * division is the floor.
 */
#define ORC_ONE ((int64_t)1 << 16)

static int64_t orc_distance(int32_t sab, int32_t saa, int32_t sbb)
{
    int64_t m = saa > sbb ? saa : sbb;
    if (m <= 0) return 0;
    return ORC_ONE - ((int64_t)sab * ORC_ONE) / m;
}

/*
 * Row sums of the exact center: rowsum[x] = sum_{r in refs} d(c_x, r) for
 * the listed candidates c_x (cands == NULL: every sequence, ncand == n),
 * where refs is every sequence (refs == NULL) or a given subset; d(i, i) = 0.
 * Returns 0, or -1 on error.
 */
int orc_center_rowsums(const uint8_t *res, const int64_t *off, int64_t n,
                       const int64_t *cands, int64_t ncand,
                       const int64_t *refs, int64_t nref,
                       const int8_t *M, int32_t K, int32_t o, int32_t e,
                       int64_t *rowsum, int threads)
{
    int64_t nc = cands ? ncand : n;
    int64_t nr = refs ? nref : n;
    int64_t np = nc * nr + n;
    int64_t *pairs = malloc(sizeof(int64_t) * 2 * np);
    int32_t *S = malloc(sizeof(int32_t) * np);
    if (!pairs || !S) { free(pairs); free(S); return -1; }
    for (int64_t x = 0; x < nc; x++)
        for (int64_t r = 0; r < nr; r++) {
            pairs[2 * (x * nr + r)] = cands ? cands[x] : x;
            pairs[2 * (x * nr + r) + 1] = refs ? refs[r] : r;
        }
    for (int64_t i = 0; i < n; i++) {          /* self scores S(i,i) */
        pairs[2 * (nc * nr + i)] = i;
        pairs[2 * (nc * nr + i) + 1] = i;
    }
    if (orc_pair_scores(res, off, pairs, np, M, K, o, e, S, threads) != 0) {
        free(pairs); free(S); return -1;
    }
    const int32_t *self = S + nc * nr;
    for (int64_t x = 0; x < nc; x++) {
        int64_t i = cands ? cands[x] : x, sum = 0;
        for (int64_t r = 0; r < nr; r++) {
            int64_t ri = refs ? refs[r] : r;
            sum += orc_distance(S[x * nr + r], self[i], self[ri]);
        }
        rowsum[x] = sum;
    }
    free(pairs); free(S);
    return 0;
}

/*
 * Exact center star: the row sums of every sequence (as orc_center_rowsums)
 * and the lowest index with the smallest one (-1 on error).
 */
int64_t orc_exact_center(const uint8_t *res, const int64_t *off, int64_t n,
                         const int64_t *refs, int64_t nref,
                         const int8_t *M, int32_t K, int32_t o, int32_t e,
                         int64_t *rowsum, int threads)
{
    int64_t *rs = rowsum ? rowsum : malloc(sizeof(int64_t) * n);
    if (!rs) return -1;
    int64_t bestc = -1;
    if (orc_center_rowsums(res, off, n, NULL, n, refs, nref, M, K, o, e, rs, threads) == 0) {
        bestc = 0;
        for (int64_t i = 1; i < n; i++)
            if (rs[i] < rs[bestc]) bestc = i;
    }
    if (!rowsum) free(rs);
    return bestc;
}

/* ====================================================================== */
/*
 * Anchored alignment of similar sequences (the paper's trie path for similar
 * nucleotides: the center's segments are indexed, matched segments of the
 * other sequence are skipped and only the unmatched stretches are aligned).
 * Reading:
 *   - segments: the center cut into S = floor(Lc / k) non-overlapping pieces
 *     c[s k .. s k + k), s = 0..S-1 (a shorter tail is no segment);
 *   - matches: every (s, p) with x[p .. p + k) equal to segment s;
 *   - chain: matches (s_1, p_1), ..., (s_T, p_T) with s increasing and
 *     p_{t+1} >= p_t + k, as many as possible; matches are ordered by (s, p)
 *     and each takes as predecessor the first compatible match (in that
 *     order) of the longest chain ending before it; the chain ends at the
 *     first match of the longest chain;
 *   - between consecutive anchors the unmatched stretches of the center and
 *     of the sequence are aligned globally (Gotoh with W_k = o + (k-1)e, the
 *     end cells' gap runs charged from the stretch's edge, traceback from the
 *     end: diagonal, then F, then E; a gap extends only when strictly
 *     better);
 *   - before the first anchor and after the last the flank rule of the local
 *     path applies (prefix right-aligned, suffix left-aligned, no gaps,
 *     surplus sequence residues in slot 0 / slot Lc);
 *   - the local path instead (the Smith-Waterman alignment, orc_sw +
 *     orc_traceback) when there is no match, when there are more matches
 *     than ORC_ANCH_CAP(S) = the smallest power of two >= max(64, 2 S), or
 *     when a stretch between consecutive anchors is longer than
 *     ORC_ANCH_BOX = 80 residues on either side (the anchored path aligns
 *     only short unmatched stretches; longer ones are left to the local
 *     alignment of the whole pair).
 * Output as orc_traceback's: ins[0..Lc], occ[0..Lc]; seg = {score, i1, j1,
 * i2, j2} with the anchored region c[i1+1..i2] x x[j1+1..j2] (first anchor's
 * start to last anchor's end) and score its affine score, or the
 * Smith-Waterman segment when there is no anchor.  Returns 0, -1 on error.
 */

/* Global affine alignment of c[0..lc) with x[0..lx); adds its columns to
 * ins/occ at center offset a (c[i] is center residue a+i+1) and returns the
 * score (INT32_MIN on error). */
static int32_t orc_global_stretch(const uint8_t *c, int32_t lc, const uint8_t *x, int32_t lx,
                                  const int8_t *M, int32_t K, int32_t o, int32_t e,
                                  int32_t a, uint16_t *ins, uint8_t *occ)
{
    if (lc == 0 && lx == 0) return 0;
    size_t w = (size_t)lx + 1, cells = ((size_t)lc + 1) * w;
    int32_t *H = malloc(cells * sizeof(int32_t));
    int32_t *E = malloc(cells * sizeof(int32_t));
    int32_t *F = malloc(cells * sizeof(int32_t));
    if (!H || !E || !F) { free(H); free(E); free(F); return INT32_MIN; }
    H[0] = 0; E[0] = ORC_NEG; F[0] = ORC_NEG;
    for (int32_t j = 1; j <= lx; j++) {       /* x residues against gaps */
        E[j] = -(o + (j - 1) * e); H[j] = E[j]; F[j] = ORC_NEG;
    }
    for (int32_t i = 1; i <= lc; i++) {       /* c residues against gaps */
        size_t at = (size_t)i * w;
        F[at] = -(o + (i - 1) * e); H[at] = F[at]; E[at] = ORC_NEG;
        for (int32_t j = 1; j <= lx; j++) {
            at = (size_t)i * w + j;
            E[at] = max2(H[at - 1] - o, E[at - 1] - e);
            F[at] = max2(H[at - w] - o, F[at - w] - e);
            H[at] = max2(H[at - w - 1] + M[c[i - 1] * K + x[j - 1]], max2(E[at], F[at]));
        }
    }
    int32_t score = H[(size_t)lc * w + lx];
    int32_t i = lc, j = lx, state = 0;  /* 0 = H, 1 = F (c residue vs gap), 2 = E (x residue inserted) */
    while (i > 0 || j > 0) {
        size_t at = (size_t)i * w + j;
        if (state == 0) {
            if (i == 0) state = 2;
            else if (j == 0) state = 1;
            else {
                int32_t dv = H[at - w - 1] + M[c[i - 1] * K + x[j - 1]];
                if (H[at] == dv) { occ[a + i] = 1; i--; j--; continue; }
                state = H[at] == F[at] ? 1 : 2;
            }
        }
        if (state == 1) {                     /* F(i,j): from F(i-1,j) - e or H(i-1,j) - o */
            int ext = i > 1 && F[at - w] - e > H[at - w] - o;
            if (j == 0) ext = i > 1;          /* the edge column is one gap run */
            i--;
            state = ext ? 1 : 0;
        } else {                              /* E(i,j): from E(i,j-1) - e or H(i,j-1) - o */
            int ext = j > 1 && E[at - 1] - e > H[at - 1] - o;
            if (i == 0) ext = j > 1;          /* the edge row is one gap run */
            ins[a + i]++;
            j--;
            state = ext ? 2 : 0;
        }
    }
    free(H); free(E); free(F);
    return score;
}

#define ORC_ANCH_BOX 80

static int64_t orc_anch_cap(int32_t S)
{
    int64_t cap = 64;
    while (cap < 2 * (int64_t)S) cap *= 2;
    return cap;
}

static int orc_local_row(const uint8_t *c, int32_t lc, const uint8_t *x, int32_t lx,
                         const int8_t *M, int32_t K, int32_t o, int32_t e,
                         uint16_t *ins, uint8_t *occ, int32_t *seg)
{
    uint8_t *codes = malloc((size_t)lc * lx + 1);
    int32_t end[2];
    if (!codes) return -1;
    int32_t best = orc_sw(c, lc, x, lx, M, K, o, e, codes, end);
    int rc = best < 0 ? -1 : orc_traceback(codes, lc, lx, best, end[0], end[1], ins, occ, seg + 1);
    seg[0] = best;
    free(codes);
    return rc;
}

int orc_anchored(const uint8_t *c, int32_t lc, const uint8_t *x, int32_t lx,
                 const int8_t *M, int32_t K, int32_t o, int32_t e, int32_t k,
                 uint16_t *ins, uint8_t *occ, int32_t *seg)
{
    memset(ins, 0, sizeof(uint16_t) * ((size_t)lc + 1));
    memset(occ, 0, (size_t)lc + 1);
    int32_t S = k > 0 ? lc / k : 0;
    /* matches in (s, p) order */
    int64_t cap = 16, nm = 0;
    int32_t *ms = malloc(sizeof(int32_t) * cap), *mp = malloc(sizeof(int32_t) * cap);
    if (!ms || !mp) { free(ms); free(mp); return -1; }
    for (int32_t s = 0; s < S; s++)
        for (int32_t p = 0; p + k <= lx; p++) {
            if (memcmp(c + (size_t)s * k, x + p, (size_t)k) != 0) continue;
            if (nm == cap) {
                cap *= 2;
                int32_t *a1 = realloc(ms, sizeof(int32_t) * cap), *a2 = realloc(mp, sizeof(int32_t) * cap);
                if (!a1 || !a2) { free(a1 ? a1 : ms); free(a2 ? a2 : mp); return -1; }
                ms = a1; mp = a2;
            }
            ms[nm] = s; mp[nm] = p; nm++;
        }
    if (nm == 0 || nm > orc_anch_cap(S)) {   /* no anchor, or too many matches: the local path */
        free(ms); free(mp);
        return orc_local_row(c, lc, x, lx, M, K, o, e, ins, occ, seg);
    }
    /* longest chain: len[m] = 1 + len of the first compatible predecessor of
     * the longest chains before it */
    int32_t *len = malloc(sizeof(int32_t) * nm), *pred = malloc(sizeof(int32_t) * nm);
    if (!len || !pred) { free(ms); free(mp); free(len); free(pred); return -1; }
    int64_t endm = 0;
    for (int64_t m = 0; m < nm; m++) {
        len[m] = 1; pred[m] = -1;
        for (int64_t q = 0; q < m; q++)
            if (ms[q] < ms[m] && mp[q] + k <= mp[m] && len[q] + 1 > len[m]) {
                len[m] = len[q] + 1; pred[m] = (int32_t)q;
            }
        if (len[m] > len[endm]) endm = m;
    }
    int32_t T = len[endm];
    int32_t *cs = malloc(sizeof(int32_t) * T), *cp = malloc(sizeof(int32_t) * T);
    if (!cs || !cp) { free(ms); free(mp); free(len); free(pred); free(cs); free(cp); return -1; }
    for (int64_t m = endm, t = T - 1; m >= 0; m = pred[m], t--) { cs[t] = ms[m]; cp[t] = mp[m]; }
    for (int32_t t = 0; t + 1 < T; t++)      /* a long stretch: the local path */
        if (cs[t + 1] * k - (cs[t] * k + k) > ORC_ANCH_BOX || cp[t + 1] - (cp[t] + k) > ORC_ANCH_BOX) {
            free(ms); free(mp); free(len); free(pred); free(cs); free(cp);
            return orc_local_row(c, lc, x, lx, M, K, o, e, ins, occ, seg);
        }
    int32_t score = 0;
    for (int32_t t = 0; t < T; t++) {
        int32_t ca = cs[t] * k, xa = cp[t];   /* anchor t: c[ca..ca+k) = x[xa..xa+k) */
        for (int32_t u = 0; u < k; u++) { occ[ca + u + 1] = 1; score += M[c[ca + u] * K + x[xa + u]]; }
        if (t + 1 < T) {                      /* the stretch up to the next anchor */
            int32_t cb = ca + k, xb = xa + k, ce = cs[t + 1] * k, xe = cp[t + 1];
            int32_t v = orc_global_stretch(c + cb, ce - cb, x + xb, xe - xb, M, K, o, e, cb, ins, occ);
            if (v == INT32_MIN) { score = INT32_MIN; break; }
            score += v;
        }
    }
    int32_t i1 = cs[0] * k, j1 = cp[0], i2 = cs[T - 1] * k + k, j2 = cp[T - 1] + k;
    free(ms); free(mp); free(len); free(pred); free(cs); free(cp);
    if (score == INT32_MIN) return -1;
    /* flanks as on the local path */
    int32_t kk = i1 < j1 ? i1 : j1;
    for (int32_t t = 0; t < kk; t++) occ[i1 - t] = 1;
    if (j1 > i1) ins[0] = (uint16_t)(ins[0] + (j1 - i1));
    int32_t ra = lc - i2, rb = lx - j2;
    kk = ra < rb ? ra : rb;
    for (int32_t t = 1; t <= kk; t++) occ[i2 + t] = 1;
    if (rb > ra) ins[lc] += (uint16_t)(rb - ra);
    seg[0] = score; seg[1] = i1; seg[2] = j1; seg[3] = i2; seg[4] = j2;
    return 0;
}

typedef struct {
    orc_seqs q; int64_t center; int32_t lc, k;
    uint16_t *ins; uint8_t *occ; int32_t *seg; atomic_int err;
} anchored_job;

static void anchored_task(void *ctx, int64_t t)
{
    anchored_job *j = ctx;
    const orc_seqs *q = &j->q;
    const uint8_t *c = q->res + q->off[j->center];
    const uint8_t *s = q->res + q->off[t];
    int32_t ls = (int32_t)(q->off[t + 1] - q->off[t]);
    if (orc_anchored(c, j->lc, s, ls, q->M, q->K, q->o, q->e, j->k,
                     j->ins + (size_t)t * (j->lc + 1), j->occ + (size_t)t * (j->lc + 1),
                     j->seg + 5 * t) != 0)
        atomic_store(&j->err, 1);
}

/* Every sequence aligned to the center by orc_anchored (rows as orc_align_all). */
int orc_anchored_all(const uint8_t *res, const int64_t *off, int64_t n, int64_t center,
                     const int8_t *M, int32_t K, int32_t o, int32_t e, int32_t k,
                     uint16_t *ins, uint8_t *occ, int32_t *seg, int threads)
{
    anchored_job j = { { res, off, M, K, o, e }, center,
                       (int32_t)(off[center + 1] - off[center]), k, ins, occ, seg, 0 };
    orc_parallel_for(n, threads, anchored_task, &j);
    return atomic_load(&j.err) ? -1 : 0;
}
