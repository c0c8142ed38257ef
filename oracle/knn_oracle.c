/*
 * CPU oracle for the sparse-vector KNN join -- TEST INFRASTRUCTURE, NOT THE PRODUCT.
 *
 * Only the tests, the package smoke check and the benchmark's CPU-baseline leg may
 * load this library.  It shares no code, header, table or helper with the CUDA
 * library; it reads the same seeded inputs and nothing else.
 *
 * Paper: Wang, Lin, Huang, Wang, He, "Efficient K-Nearest Neighbor Join Algorithms
 * for High Dimensional Sparse Data".
 *
 *   oracle_bf_join    The plain definition of the result (Section 3): for every r,
 *                     dot(r,s) of eq. (1) for every s, computed by the two-pointer
 *                     merge of Algorithm 2 (function dot); keep the s with a positive
 *                     score, order them by (score desc, s id asc), emit the first k.
 *   oracle_iib_join   Algorithm 3 (IIB) run inside the block nested loop join of
 *                     Algorithm 1: per (R block, S block) build the inverted lists,
 *                     then Find_Matches_IIB for every r of the R block.
 *   oracle_iiib_join  Algorithm 4 (IIIB) inside Algorithm 1: per (R block, S block)
 *                     reorder the dimensions by frequency in the R block, take
 *                     maxWeight_d over the R block and MinPruneScore = min pruneScore,
 *                     index each s only from the feature where the running bound t
 *                     exceeds MinPruneScore, then Find_Matches_IIIB (scan the reduced
 *                     lists, complete every non-zero score with dot over the
 *                     unindexed features, insert when above pruneScore).
 *
 * Arithmetic: every weight is widened to double and every score is a double sum.  For
 * uint8 inputs every product and partial sum is an integer below 2^53, so the double
 * result is the exact integer; for float32 inputs this is the fp64 reference.
 *
 * Readings of points the paper leaves open (each is also listed in the design notes):
 *   - "For each s with non-zero score in A" visits s in ascending id, and the strict
 *     "A[s] > pruneScore(r)" therefore keeps the lower id among equal scores, which
 *     is the (score desc, id asc) order of the plain definition.
 *   - pruneScore(r) is 0 until the candidate set holds k vectors, then the k-th score.
 *   - Insertion places a new vector after the candidates whose score equals its own.
 *   - Algorithm 4 ties in the frequency order are broken by ascending dimension.
 *   - Zero scores never enter the result; rows with fewer than k positive scores are
 *     padded with id -1 and score 0.
 *
 * Parity is pinned by tests (hand-worked examples, a dense int64 matmul with a stable
 * sort, brute force on tiny inputs, Theorem 1 equivalences, posting-count invariants).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int64_t n_rows;
    int32_t dim;
    const int64_t* indptr;   /* [n_rows+1] */
    const int32_t* indices;  /* [nnz], ascending within each row */
    const void* values;      /* [nnz] uint8 or float32 */
    int32_t dtype;           /* 0 = uint8, 1 = float32 */
} ocsr;

typedef struct {
    int64_t postings_touched;  /* score updates in Find_Matches (Algorithms 3, 4)      */
    int64_t postings_indexed;  /* pairs inserted into inverted lists                    */
    int64_t merge_steps;       /* loop iterations of dot() (eq. 2 / eq. 3 cost)          */
    int64_t residual_dots;     /* calls of dot() on the unindexed remainder (Alg. 4)     */
} ostats;

static double wval(const ocsr* x, int64_t j) {
    if (x->dtype == 0) return (double)((const uint8_t*)x->values)[j];
    return (double)((const float*)x->values)[j];
}

/* ------------------------------------------------------------------------------- */
/* dot(r, s): Algorithm 2, function dot -- two iterators advance over the ascending */
/* features; equal dimensions contribute w_r * w_s.  `skip` (may be NULL) marks s   */
/* features that Algorithm 4 has removed from s after indexing them.              */
/* ------------------------------------------------------------------------------- */
static double dot_merge(const ocsr* R, int64_t r, const ocsr* S, int64_t s,
                        const unsigned char* skip, int64_t* steps) {
    double ret = 0.0;
    int64_t i = R->indptr[r], ie = R->indptr[r + 1];
    int64_t j = S->indptr[s], je = S->indptr[s + 1];
    int64_t n = 0;
    while (i < ie && j < je) {
        if (skip && skip[j - S->indptr[0]]) { j++; continue; }
        int32_t dr = R->indices[i], ds = S->indices[j];
        n++;
        if (dr == ds) {
            ret += wval(R, i) * wval(S, j);
            i++; j++;
        } else if (dr > ds) {
            j++;
        } else {
            i++;
        }
    }
    if (steps) *steps += n;
    return ret;
}

/* ------------------------------------------------------------------------------- */
/* Plain definition                                                                 */
/* ------------------------------------------------------------------------------- */
typedef struct { double score; int64_t id; } pair_t;

static int cmp_pair(const void* a, const void* b) {
    const pair_t* x = (const pair_t*)a;
    const pair_t* y = (const pair_t*)b;
    if (x->score > y->score) return -1;
    if (x->score < y->score) return 1;
    if (x->id < y->id) return -1;
    if (x->id > y->id) return 1;
    return 0;
}

int oracle_bf_join(const ocsr* R, const ocsr* S, int32_t k, int32_t nthreads,
                   int32_t* out_ids, double* out_scores, ostats* st) {
    if (k < 1) return 1;
    int64_t steps_total = 0;
#ifdef _OPENMP
    omp_set_num_threads(nthreads > 0 ? nthreads : omp_get_num_procs());   // 0: every host core
#endif
#pragma omp parallel reduction(+ : steps_total)
    {
        pair_t* all = (pair_t*)malloc(sizeof(pair_t) * (size_t)(S->n_rows > 0 ? S->n_rows : 1));
#pragma omp for schedule(dynamic, 1)
        for (int64_t r = 0; r < R->n_rows; r++) {
            int64_t m = 0;
            for (int64_t s = 0; s < S->n_rows; s++) {
                double v = dot_merge(R, r, S, s, NULL, &steps_total);
                if (v > 0.0) { all[m].score = v; all[m].id = s; m++; }
            }
            qsort(all, (size_t)m, sizeof(pair_t), cmp_pair);
            for (int32_t q = 0; q < k; q++) {
                out_ids[r * k + q] = q < m ? (int32_t)all[q].id : -1;
                out_scores[r * k + q] = q < m ? all[q].score : 0.0;
            }
        }
        free(all);
    }
    if (st) { memset(st, 0, sizeof(*st)); st->merge_steps = steps_total; }
    return 0;
}

/* ------------------------------------------------------------------------------- */
/* KNN candidate set of one r and its pruneScore (Algorithms 2 and 3)             */
/* ------------------------------------------------------------------------------- */
typedef struct { int32_t k, size; int64_t* id; double* sc; } cand_t;

static double prune_score(const cand_t* c) { return c->size == c->k ? c->sc[c->k - 1] : 0.0; }

static void cand_insert(cand_t* c, int64_t s, double v) {
    int32_t p = 0;
    while (p < c->size && c->sc[p] >= v) p++;   /* after equal scores */
    if (p >= c->k) return;
    int32_t last = c->size < c->k ? c->size : c->k - 1;
    for (int32_t q = last; q > p; q--) { c->sc[q] = c->sc[q - 1]; c->id[q] = c->id[q - 1]; }
    c->sc[p] = v; c->id[p] = s;
    if (c->size < c->k) c->size++;
}

/* Inverted lists of one S block: for each d, the pairs (s, w) with w = s[d] != 0.  */
typedef struct { int64_t* off; int64_t* sid; double* w; } inv_t;

static void inv_alloc(inv_t* I, int32_t dim, int64_t cap) {
    I->off = (int64_t*)calloc((size_t)dim + 1, sizeof(int64_t));
    I->sid = (int64_t*)malloc(sizeof(int64_t) * (size_t)(cap > 0 ? cap : 1));
    I->w = (double*)malloc(sizeof(double) * (size_t)(cap > 0 ? cap : 1));
}
static void inv_free(inv_t* I) { free(I->off); free(I->sid); free(I->w); }

/* Create_Inverted_List_IIB (Algorithm 3): s in ascending order, every
 * feature (d, w) of s appended to I_d.  Built as counts then fills.                */
static void create_inverted_list_iib(const ocsr* S, int64_t s0, int64_t s1, inv_t* I,
                                     int64_t* n_indexed) {
    int32_t D = S->dim;
    memset(I->off, 0, sizeof(int64_t) * ((size_t)D + 1));
    for (int64_t j = S->indptr[s0]; j < S->indptr[s1]; j++) I->off[S->indices[j] + 1]++;
    for (int32_t d = 0; d < D; d++) I->off[d + 1] += I->off[d];
    int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)(D > 0 ? D : 1));
    memcpy(fill, I->off, sizeof(int64_t) * (size_t)D);
    for (int64_t s = s0; s < s1; s++)
        for (int64_t j = S->indptr[s]; j < S->indptr[s + 1]; j++) {
            int32_t d = S->indices[j];
            I->sid[fill[d]] = s; I->w[fill[d]] = wval(S, j); fill[d]++;
        }
    *n_indexed += S->indptr[s1] - S->indptr[s0];
    free(fill);
}

int oracle_iib_join(const ocsr* R, const ocsr* S, int32_t k, int64_t rblock, int64_t sblock,
                    int32_t nthreads, int32_t* out_ids, double* out_scores, ostats* st) {
    if (k < 1) return 1;
    if (rblock <= 0) rblock = R->n_rows > 0 ? R->n_rows : 1;
    if (sblock <= 0) sblock = S->n_rows > 0 ? S->n_rows : 1;
#ifdef _OPENMP
    omp_set_num_threads(nthreads > 0 ? nthreads : omp_get_num_procs());   // 0: every host core
#endif
    ostats acc; memset(&acc, 0, sizeof(acc));
    inv_t I; inv_alloc(&I, S->dim, S->indptr[S->n_rows] - S->indptr[0]);
    int64_t* cid = (int64_t*)malloc(sizeof(int64_t) * (size_t)(rblock * k));
    double* csc = (double*)malloc(sizeof(double) * (size_t)(rblock * k));
    int32_t* csize = (int32_t*)malloc(sizeof(int32_t) * (size_t)rblock);

    /* Algorithm 1: each R block, then each S block in order */
    for (int64_t r0 = 0; r0 < R->n_rows; r0 += rblock) {
        int64_t r1 = r0 + rblock < R->n_rows ? r0 + rblock : R->n_rows;
        for (int64_t q = 0; q < r1 - r0; q++) csize[q] = 0;   /* InitPruneScore */
        for (int64_t s0 = 0; s0 < S->n_rows; s0 += sblock) {
            int64_t s1 = s0 + sblock < S->n_rows ? s0 + sblock : S->n_rows;
            create_inverted_list_iib(S, s0, s1, &I, &acc.postings_indexed);
            int64_t touched = 0;
#pragma omp parallel reduction(+ : touched)
            {
                double* A = (double*)calloc((size_t)(s1 - s0), sizeof(double));
#pragma omp for schedule(dynamic, 1)
                for (int64_t r = r0; r < r1; r++) {   /* Find_Matches_IIB(r) */
                    cand_t c = {k, csize[r - r0], cid + (r - r0) * k, csc + (r - r0) * k};
                    for (int64_t i = R->indptr[r]; i < R->indptr[r + 1]; i++) {
                        int32_t d = R->indices[i];
                        double rw = wval(R, i);
                        for (int64_t p = I.off[d]; p < I.off[d + 1]; p++) {
                            A[I.sid[p] - s0] += rw * I.w[p];
                            touched++;
                        }
                    }
                    for (int64_t s = s0; s < s1; s++) {
                        if (A[s - s0] != 0.0) {
                            if (A[s - s0] > prune_score(&c)) cand_insert(&c, s, A[s - s0]);
                            A[s - s0] = 0.0;
                        }
                    }
                    csize[r - r0] = c.size;
                }
                free(A);
            }
            acc.postings_touched += touched;
        }
        for (int64_t r = r0; r < r1; r++)   /* OutputKNN */
            for (int32_t q = 0; q < k; q++) {
                int ok = q < csize[r - r0];
                out_ids[r * k + q] = ok ? (int32_t)cid[(r - r0) * k + q] : -1;
                out_scores[r * k + q] = ok ? csc[(r - r0) * k + q] : 0.0;
            }
    }
    free(cid); free(csc); free(csize); inv_free(&I);
    if (st) *st = acc;
    return 0;
}

/* ------------------------------------------------------------------------------- */
/* IIIB                                                                             */
/* ------------------------------------------------------------------------------- */
static int cmp_by_rank(const void* a, const void* b) {
    int64_t x = *(const int64_t*)a, y = *(const int64_t*)b;  /* packed (rank<<32)|pos */
    return x < y ? -1 : (x > y ? 1 : 0);
}

int oracle_iiib_join(const ocsr* R, const ocsr* S, int32_t k, int64_t rblock, int64_t sblock,
                     int32_t nthreads, int32_t* out_ids, double* out_scores, ostats* st) {
    if (k < 1) return 1;
    if (rblock <= 0) rblock = R->n_rows > 0 ? R->n_rows : 1;
    if (sblock <= 0) sblock = S->n_rows > 0 ? S->n_rows : 1;
#ifdef _OPENMP
    omp_set_num_threads(nthreads > 0 ? nthreads : omp_get_num_procs());   // 0: every host core
#endif
    int32_t D = S->dim;
    ostats acc; memset(&acc, 0, sizeof(acc));
    int64_t nnzS = S->indptr[S->n_rows] - S->indptr[0];
    inv_t I; inv_alloc(&I, D, nnzS);
    int64_t* cid = (int64_t*)malloc(sizeof(int64_t) * (size_t)(rblock * k));
    double* csc = (double*)malloc(sizeof(double) * (size_t)(rblock * k));
    int32_t* csize = (int32_t*)malloc(sizeof(int32_t) * (size_t)rblock);
    int64_t* freq = (int64_t*)malloc(sizeof(int64_t) * (size_t)(D > 0 ? D : 1));
    double* maxw = (double*)malloc(sizeof(double) * (size_t)(D > 0 ? D : 1));
    int32_t* rank = (int32_t*)malloc(sizeof(int32_t) * (size_t)(D > 0 ? D : 1));
    int64_t* order = (int64_t*)malloc(sizeof(int64_t) * (size_t)(D > 0 ? D : 1));
    unsigned char* removed = (unsigned char*)malloc((size_t)(nnzS > 0 ? nnzS : 1));
    int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)(D > 0 ? D : 1));
    int64_t maxnnz = 1;
    for (int64_t s = 0; s < S->n_rows; s++)
        if (S->indptr[s + 1] - S->indptr[s] > maxnnz) maxnnz = S->indptr[s + 1] - S->indptr[s];
    int64_t* feat = (int64_t*)malloc(sizeof(int64_t) * (size_t)maxnnz);
    int64_t j0 = S->indptr[0];

    for (int64_t r0 = 0; r0 < R->n_rows; r0 += rblock) {
        int64_t r1 = r0 + rblock < R->n_rows ? r0 + rblock : R->n_rows;
        for (int64_t q = 0; q < r1 - r0; q++) csize[q] = 0;   /* InitPruneScore */

        /* Algorithm 4: dimensions with more non-zero entries in B_r come first (ties:
         * ascending d), and maxWeight_d(B_r).  Both depend on B_r only.           */
        for (int32_t d = 0; d < D; d++) { freq[d] = 0; maxw[d] = 0.0; }
        for (int64_t i = R->indptr[r0]; i < R->indptr[r1]; i++) {
            int32_t d = R->indices[i];
            if (d < 0 || d >= D) continue;
            freq[d]++;
            if (wval(R, i) > maxw[d]) maxw[d] = wval(R, i);
        }
        /* order = dimensions sorted by (freq desc, d asc); rank = inverse order */
        {
            int64_t* keys = order;
            int64_t maxf = (r1 - r0) + 1;
            for (int32_t d = 0; d < D; d++) keys[d] = ((maxf - freq[d]) << 32) | (int64_t)d;
            qsort(keys, (size_t)D, sizeof(int64_t), cmp_by_rank);
            for (int32_t p = 0; p < D; p++) rank[keys[p] & 0xffffffff] = p;
        }

        for (int64_t s0 = 0; s0 < S->n_rows; s0 += sblock) {
            int64_t s1 = s0 + sblock < S->n_rows ? s0 + sblock : S->n_rows;
            /* MinPruneScore = min over B_r of pruneScore(r), from earlier S blocks */
            double mps = 0.0;
            for (int64_t r = r0; r < r1; r++) {
                double p = csize[r - r0] == k ? csc[(r - r0) * k + k - 1] : 0.0;
                if (r == r0 || p < mps) mps = p;
            }
            /* Create_Inverted_List_IIIB (Algorithm 4).  A fresh ReadBlock of the S
             * block (Algorithm 1) restores every feature of s.                       */
            memset(I.off, 0, sizeof(int64_t) * ((size_t)D + 1));
            for (int64_t s = s0; s < s1; s++) {
                int64_t a = S->indptr[s], b = S->indptr[s + 1];
                for (int64_t j = a; j < b; j++)
                    feat[j - a] = ((int64_t)rank[S->indices[j]] << 32) | (j - a);
                qsort(feat, (size_t)(b - a), sizeof(int64_t), cmp_by_rank);
                double t = 0.0;
                for (int64_t q = 0; q < b - a; q++) {
                    int64_t j = a + (feat[q] & 0xffffffff);
                    int32_t d = S->indices[j];
                    t += maxw[d] * wval(S, j);
                    if (t > mps) { removed[j - j0] = 1; I.off[d + 1]++; }
                    else removed[j - j0] = 0;
                }
            }
            for (int32_t d = 0; d < D; d++) I.off[d + 1] += I.off[d];
            memcpy(fill, I.off, sizeof(int64_t) * (size_t)D);
            for (int64_t s = s0; s < s1; s++)
                for (int64_t j = S->indptr[s]; j < S->indptr[s + 1]; j++)
                    if (removed[j - j0]) {
                        int32_t d = S->indices[j];
                        I.sid[fill[d]] = s; I.w[fill[d]] = wval(S, j); fill[d]++;
                    }
            acc.postings_indexed += I.off[D];

            int64_t touched = 0, steps = 0, rdots = 0;
#pragma omp parallel reduction(+ : touched, steps, rdots)
            {
                double* A = (double*)calloc((size_t)(s1 - s0), sizeof(double));
#pragma omp for schedule(dynamic, 1)
                for (int64_t r = r0; r < r1; r++) {   /* Find_Matches_IIIB(r) */
                    cand_t c = {k, csize[r - r0], cid + (r - r0) * k, csc + (r - r0) * k};
                    for (int64_t i = R->indptr[r]; i < R->indptr[r + 1]; i++) {
                        int32_t d = R->indices[i];
                        double rw = wval(R, i);
                        for (int64_t p = I.off[d]; p < I.off[d + 1]; p++) {
                            A[I.sid[p] - s0] += rw * I.w[p];
                            touched++;
                        }
                    }
                    for (int64_t s = s0; s < s1; s++) {
                        if (A[s - s0] != 0.0) {
                            /* completion: dot over the remaining (unindexed) features of s */
                            double v = A[s - s0] + dot_merge(R, r, S, s, removed, &steps);
                            rdots++;
                            if (v > prune_score(&c)) cand_insert(&c, s, v);
                            A[s - s0] = 0.0;
                        }
                    }
                    csize[r - r0] = c.size;
                }
                free(A);
            }
            acc.postings_touched += touched;
            acc.merge_steps += steps;
            acc.residual_dots += rdots;
        }
        for (int64_t r = r0; r < r1; r++)   /* OutputKNN */
            for (int32_t q = 0; q < k; q++) {
                int ok = q < csize[r - r0];
                out_ids[r * k + q] = ok ? (int32_t)cid[(r - r0) * k + q] : -1;
                out_scores[r * k + q] = ok ? csc[(r - r0) * k + q] : 0.0;
            }
    }
    free(cid); free(csc); free(csize); free(freq); free(maxw); free(rank); free(order);
    free(removed); free(fill); free(feat); inv_free(&I);
    if (st) *st = acc;
    return 0;
}
