/*
 * SubQuad all-candidates affinity stage -- the ORACLE.
 *
 * This file is test infrastructure.  It is a plain, slow, single-threaded C
 * restatement of what the method computes, written from the paper and the
 * readings listed with each function, in FP64 wherever the quantity is
 * floating point.  Only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg load it; the library path never does, and it shares no
 * code, header, table or helper with the CUDA sources.
 *
 * Notation: n sequences s_i of length L_i over the 20 amino acids (codes 0..19
 * in the order ACDEFGHIKLMNPQRSTVWY), H hash functions grouped into B bands of
 * R rows, candidate set C of unordered pairs (i < j).
 *
 * Parity status: every function below is pinned by tests against something
 * other than itself (hand-worked alignments, brute-force enumeration,
 * textbook reductions, library routines, statistical bounds, finite
 * differences); the pin is named beside each function.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define P31 2147483647ULL /* 2^31 - 1 */

/* ------------------------------------------------------------------------- */
/* BLOSUM62 (Henikoff & Henikoff 1992), transcribed in the customary NCBI row
 * order ARNDCQEGHILKMFPSTWYV and re-indexed to the alphabetical code order.
 * Pins: symmetry, diagonal strict row maximum, spot entries, and a
 * cell-by-cell comparison with the library's separately typed table.        */
/* ------------------------------------------------------------------------- */
static const char NCBI_ORDER[21] = "ARNDCQEGHILKMFPSTWYV";
static const char CODE_ORDER[21] = "ACDEFGHIKLMNPQRSTVWY";
static const int BLOSUM62_NCBI[20][20] = {
    /*        A   R   N   D   C   Q   E   G   H   I   L   K   M   F   P   S   T   W   Y   V */
    /* A */ { 4, -1, -2, -2,  0, -1, -1,  0, -2, -1, -1, -1, -1, -2, -1,  1,  0, -3, -2,  0},
    /* R */ {-1,  5,  0, -2, -3,  1,  0, -2,  0, -3, -2,  2, -1, -3, -2, -1, -1, -3, -2, -3},
    /* N */ {-2,  0,  6,  1, -3,  0,  0,  0,  1, -3, -3,  0, -2, -3, -2,  1,  0, -4, -2, -3},
    /* D */ {-2, -2,  1,  6, -3,  0,  2, -1, -1, -3, -4, -1, -3, -3, -1,  0, -1, -4, -3, -3},
    /* C */ { 0, -3, -3, -3,  9, -3, -4, -3, -3, -1, -1, -3, -1, -2, -3, -1, -1, -2, -2, -1},
    /* Q */ {-1,  1,  0,  0, -3,  5,  2, -2,  0, -3, -2,  1,  0, -3, -1,  0, -1, -2, -1, -2},
    /* E */ {-1,  0,  0,  2, -4,  2,  5, -2,  0, -3, -3,  1, -2, -3, -1,  0, -1, -3, -2, -2},
    /* G */ { 0, -2,  0, -1, -3, -2, -2,  6, -2, -4, -4, -2, -3, -3, -2,  0, -2, -2, -3, -3},
    /* H */ {-2,  0,  1, -1, -3,  0,  0, -2,  8, -3, -3, -1, -2, -1, -2, -1, -2, -2,  2, -3},
    /* I */ {-1, -3, -3, -3, -1, -3, -3, -4, -3,  4,  2, -3,  1,  0, -3, -2, -1, -3, -1,  3},
    /* L */ {-1, -2, -3, -4, -1, -2, -3, -4, -3,  2,  4, -2,  2,  0, -3, -2, -1, -2, -1,  1},
    /* K */ {-1,  2,  0, -1, -3,  1,  1, -2, -1, -3, -2,  5, -1, -3, -1,  0, -1, -3, -2, -2},
    /* M */ {-1, -1, -2, -3, -1,  0, -2, -3, -2,  1,  2, -1,  5,  0, -2, -1, -1, -1, -1,  1},
    /* F */ {-2, -3, -3, -3, -2, -3, -3, -3, -1,  0,  0, -3,  0,  6, -4, -2, -2,  1,  3, -1},
    /* P */ {-1, -2, -2, -1, -3, -1, -1, -2, -2, -3, -3, -1, -2, -4,  7, -1, -1, -4, -3, -2},
    /* S */ { 1, -1,  1,  0, -1,  0,  0,  0, -1, -2, -2,  0, -1, -2, -1,  4,  1, -3, -2, -2},
    /* T */ { 0, -1,  0, -1, -1, -1, -1, -2, -2, -1, -1, -1, -1, -2, -1,  1,  5, -2, -2,  0},
    /* W */ {-3, -3, -4, -4, -2, -2, -3, -2, -2, -3, -2, -3, -1,  1, -4, -3, -2, 11,  2, -3},
    /* Y */ {-2, -2, -2, -3, -2, -1, -2, -3,  2, -1, -1, -2, -1,  3, -3, -2, -2,  2,  7, -1},
    /* V */ { 0, -3, -3, -3, -1, -2, -2, -3, -3,  3,  1, -2,  1, -1, -2, -2,  0, -3, -1,  4},
};

static int ncbi_index(char letter)
{
    for (int r = 0; r < 20; ++r)
        if (NCBI_ORDER[r] == letter) return r;
    return -1;
}

/* out[20*a + b] = BLOSUM62(letter a, letter b), a, b in code order. */
void oracle_blosum62(int32_t *out)
{
    for (int a = 0; a < 20; ++a)
        for (int b = 0; b < 20; ++b)
            out[20 * a + b] = BLOSUM62_NCBI[ncbi_index(CODE_ORDER[a])][ncbi_index(CODE_ORDER[b])];
}

/* ------------------------------------------------------------------------- */
/* MinHash signatures (Algorithm 1, preprocessing; sketch size M = H; the
 * sampling-error discussion of the appendix "Sampling Error Bounds").
 * Readings: the set of a sequence is its set of overlapping k-mers; a k-mer is
 * the base-20 integer x = sum_m code(s[p+m]) * 20^(k-1-m); hash t is
 * h_t(x) = (a_t x + b_t) mod (2^31 - 1); sig[i][t] = min over the k-mers of s_i.
 * Pins: brute-force min over k-mers in a test; collision rate against exact
 * k-mer Jaccard within the binomial error of the appendix bound.             */
/* ------------------------------------------------------------------------- */
uint64_t oracle_kmer_code(const uint8_t *s, int k)
{
    uint64_t x = 0;
    for (int m = 0; m < k; ++m) x = x * 20u + s[m];
    return x;
}

void oracle_sign(const uint8_t *codes, int code_stride, const uint8_t *lens, int64_t n, int k, int H,
                 const uint32_t *a, const uint32_t *b, uint32_t *sig /* [n][H] */)
{
    for (int64_t i = 0; i < n; ++i) {
        const uint8_t *s = codes + i * (int64_t)code_stride;
        int L = lens[i];
        for (int t = 0; t < H; ++t) {
            uint64_t best = UINT64_MAX;
            for (int p = 0; p + k <= L; ++p) {
                uint64_t x = oracle_kmer_code(s + p, k);
                uint64_t h = ((uint64_t)a[t] * x + (uint64_t)b[t]) % P31;
                if (h < best) best = h;
            }
            sig[i * H + t] = (uint32_t)best; /* L >= k is a precondition */
        }
    }
}

/* ------------------------------------------------------------------------- */
/* LSH banding and candidate list CAND (Algorithm 1, preprocessing; the index
 * of "Optimized Indexing Mechanism"; the candidate set C of the complexity
 * appendix).  Readings: band b is hash rows b*R .. b*R+R-1; its key is the
 * exact R-tuple; a bucket is the set of sequences with one key; its members,
 * ranked by ascending id, fall into chunks of `cap` consecutive ranks
 * (cap <= 0: one chunk); C is the set of pairs i < j that share a chunk in at
 * least one band.  Pin: brute-force pair test of this definition in a test.  */
/* ------------------------------------------------------------------------- */
typedef struct {
    uint32_t key[8];
    uint32_t id;
} band_rec;

static int g_rows; /* qsort has no context argument: set before any sort, never changed during one */

static int cmp_band_rec(const void *pa, const void *pb)
{
    const band_rec *x = (const band_rec *)pa, *y = (const band_rec *)pb;
    for (int r = 0; r < g_rows; ++r) {
        if (x->key[r] < y->key[r]) return -1;
        if (x->key[r] > y->key[r]) return 1;
    }
    return (x->id > y->id) - (x->id < y->id);
}

static int cmp_u64(const void *pa, const void *pb)
{
    uint64_t x = *(const uint64_t *)pa, y = *(const uint64_t *)pb;
    return (x > y) - (x < y);
}

typedef struct {
    uint64_t *v;
    int64_t len, cap;
} u64vec;

static int u64vec_push(u64vec *vec, uint64_t x)
{
    if (vec->len == vec->cap) {
        int64_t nc = vec->cap ? 2 * vec->cap : 1024;
        uint64_t *nv = (uint64_t *)realloc(vec->v, (size_t)nc * sizeof(uint64_t));
        if (!nv) return -1;
        vec->v = nv;
        vec->cap = nc;
    }
    vec->v[vec->len++] = x;
    return 0;
}

/* Appends the pairs (i << 32 | j) of every chunk of bands 0 .. bands-1 of
 * sig to *all, duplicates included; g_rows must equal rows.  Returns 0, or -1
 * on allocation failure. */
static int band_chunk_pairs(const uint32_t *sig, int64_t n, int H, int bands, int rows, int cap, u64vec *all)
{
    band_rec *recs = (band_rec *)malloc((size_t)(n > 0 ? n : 1) * sizeof(band_rec));
    if (!recs) return -1;
    for (int b = 0; b < bands; ++b) {
        for (int64_t i = 0; i < n; ++i) {
            memset(recs[i].key, 0, sizeof(recs[i].key));
            for (int r = 0; r < rows; ++r) recs[i].key[r] = sig[i * H + b * rows + r];
            recs[i].id = (uint32_t)i;
        }
        qsort(recs, (size_t)n, sizeof(band_rec), cmp_band_rec);
        int64_t s = 0;
        while (s < n) {
            int64_t e = s + 1;
            while (e < n && memcmp(recs[e].key, recs[s].key, sizeof(uint32_t) * (size_t)rows) == 0) ++e;
            for (int64_t u = s; u < e; ++u)
                for (int64_t v = u + 1; v < e; ++v) {
                    int same_chunk = cap <= 0 || ((u - s) / cap == (v - s) / cap);
                    if (same_chunk && u64vec_push(all, ((uint64_t)recs[u].id << 32) | recs[v].id) != 0) {
                        free(recs);
                        return -1;
                    }
                }
            s = e;
        }
    }
    free(recs);
    return 0;
}

/* The pairs of *all sorted, duplicates dropped, written to out (at most
 * out_capacity); returns their count.  Frees all->v. */
static int64_t sorted_unique_pairs(u64vec *all, uint32_t *out, int64_t out_capacity)
{
    if (all->len > 0) qsort(all->v, (size_t)all->len, sizeof(uint64_t), cmp_u64);
    int64_t count = 0;
    for (int64_t q = 0; q < all->len; ++q) {
        if (q > 0 && all->v[q] == all->v[q - 1]) continue;
        if (count < out_capacity) {
            out[2 * count] = (uint32_t)(all->v[q] >> 32);
            out[2 * count + 1] = (uint32_t)(all->v[q] & 0xffffffffu);
        }
        ++count;
    }
    free(all->v);
    all->v = NULL;
    return count;
}

/* Returns |C| (or -1 on allocation failure); writes min(|C|, out_capacity)
 * pairs, lexicographically sorted, as out[2q] = i, out[2q+1] = j. */
int64_t oracle_candidates(const uint32_t *sig /* [n][H] */, int64_t n, int H, int bands, int rows,
                          int cap, uint32_t *out, int64_t out_capacity)
{
    if (rows < 1 || rows > 8 || bands * rows > H) return -1;
    u64vec all = {0, 0, 0};
    g_rows = rows;
    if (band_chunk_pairs(sig, n, H, bands, rows, cap, &all) != 0) {
        free(all.v);
        return -1;
    }
    return sorted_unique_pairs(&all, out, out_capacity);
}

/* ------------------------------------------------------------------------- */
/* Affine-gap local alignment (Smith-Waterman with Gotoh's three matrices) --
 * the alignment channel a^(1) of Algorithm 1's affinity computation.
 * Reading: a gap of length l costs o + (l-1) e.  For i = 1..La, j = 1..Lb:
 *   E(i,j) = max(E(i,j-1) - e, H(i,j-1) - o)          gap in a (b_j unpaired)
 *   F(i,j) = max(F(i-1,j) - e, H(i-1,j) - o)          gap in b (a_i unpaired)
 *   H(i,j) = max(0, H(i-1,j-1) + M[a_i][b_j], E(i,j), F(i,j))
 * with H(0,.) = H(.,0) = 0 and E(.,0) = F(0,.) = -2^20; score = max H.
 * Pins: hand-worked alignments (tests/golden), exhaustive enumeration of all
 * local alignments of short strings, Kadane reduction (infinite gaps),
 * longest-common-substring reduction (identity matrix), self-score identity. */
/* ------------------------------------------------------------------------- */
#define SW_NEG (-(1 << 20))
#define SW_MAXL 64

int32_t oracle_sw(const uint8_t *a, int La, const uint8_t *b, int Lb, const int32_t *M /* [20][20] */,
                  int o, int e)
{
    int32_t Hm[SW_MAXL + 1][SW_MAXL + 1], Em[SW_MAXL + 1][SW_MAXL + 1], Fm[SW_MAXL + 1][SW_MAXL + 1];
    if (La > SW_MAXL || Lb > SW_MAXL || La < 0 || Lb < 0) return -1;
    int32_t best = 0;
    for (int i = 0; i <= La; ++i) {
        Hm[i][0] = 0;
        Em[i][0] = SW_NEG;
    }
    for (int j = 0; j <= Lb; ++j) {
        Hm[0][j] = 0;
        Fm[0][j] = SW_NEG;
    }
    for (int i = 1; i <= La; ++i)
        for (int j = 1; j <= Lb; ++j) {
            int32_t ee = Em[i][j - 1] - e, eo = Hm[i][j - 1] - o;
            int32_t ff = Fm[i - 1][j] - e, fo = Hm[i - 1][j] - o;
            Em[i][j] = ee > eo ? ee : eo;
            Fm[i][j] = ff > fo ? ff : fo;
            int32_t h = Hm[i - 1][j - 1] + M[20 * a[i - 1] + b[j - 1]];
            if (Em[i][j] > h) h = Em[i][j];
            if (Fm[i][j] > h) h = Fm[i][j];
            if (h < 0) h = 0;
            Hm[i][j] = h;
            if (h > best) best = h;
        }
    return best;
}

/* scores[p] = S(s_pairs[2p], s_pairs[2p+1]) */
void oracle_sw_pairs(const uint8_t *codes, int code_stride, const uint8_t *lens, const uint32_t *pairs,
                     int64_t m, const int32_t *M, int o, int e, int32_t *scores)
{
    for (int64_t p = 0; p < m; ++p) {
        uint32_t i = pairs[2 * p], j = pairs[2 * p + 1];
        scores[p] = oracle_sw(codes + (int64_t)i * code_stride, lens[i], codes + (int64_t)j * code_stride,
                              lens[j], M, o, e);
    }
}

/* ------------------------------------------------------------------------- */
/* Edit distance (the GPU appendix's edit-distance kernel, Eq. d_{x,y}):
 *   d(x, y) = min( d(x-1, y) + del, d(x, y-1) + ins,
 *                  d(x-1, y-1) + [a_x != b_y] sub(a_x, b_y) ),
 * d(0, 0) = 0, d(x, 0) = x del, d(0, y) = y ins; the distance is d(La, Lb).
 * Reading: insertion and deletion cost the same `indel`; the substitution cost
 * is a caller-supplied 20 x 20 table (zero on the diagonal); the default
 * "biochemical similarity" costs, in half units with indel = 2, are 1 for a
 * conservative substitution (BLOSUM62 entry > 0) and 2 otherwise -- so in the
 * paper's units an indel costs 1, a dissimilar substitution 1 and a similar
 * one 1/2.
 * Pins: hand-worked distances (tests/golden), brute-force enumeration of edit
 * scripts on short strings, Hamming distance when indels are prohibitive,
 * indel (La + Lb - 2 LCS) when substitutions are, metric axioms.           */
/* ------------------------------------------------------------------------- */
#define ED_MAXL 64

int32_t oracle_edit(const uint8_t *a, int La, const uint8_t *b, int Lb, int indel, const uint8_t *sub /* [20][20] */)
{
    int32_t D[ED_MAXL + 1][ED_MAXL + 1];
    if (La < 0 || Lb < 0 || La > ED_MAXL || Lb > ED_MAXL) return -1;
    for (int x = 0; x <= La; ++x) D[x][0] = x * indel;
    for (int y = 0; y <= Lb; ++y) D[0][y] = y * indel;
    for (int x = 1; x <= La; ++x)
        for (int y = 1; y <= Lb; ++y) {
            int32_t best = D[x - 1][y] + indel;                         /* delete a_x */
            if (D[x][y - 1] + indel < best) best = D[x][y - 1] + indel; /* insert b_y */
            int32_t diag = D[x - 1][y - 1] + (a[x - 1] != b[y - 1] ? (int32_t)sub[20 * a[x - 1] + b[y - 1]] : 0);
            if (diag < best) best = diag;
            D[x][y] = best;
        }
    return D[La][Lb];
}

void oracle_edit_pairs(const uint8_t *codes, int code_stride, const uint8_t *lens, const uint32_t *pairs, int64_t m,
                       int indel, const uint8_t *sub, int32_t *dist)
{
    for (int64_t p = 0; p < m; ++p) {
        uint32_t i = pairs[2 * p], j = pairs[2 * p + 1];
        dist[p] = oracle_edit(codes + (int64_t)i * code_stride, lens[i], codes + (int64_t)j * code_stride, lens[j],
                              indel, sub);
    }
}

/* The default substitution costs above (half units): 0 on the diagonal, 1
 * where BLOSUM62 > 0, 2 elsewhere.                                          */
void oracle_default_edit_costs(uint8_t *out /* [20][20] */)
{
    int32_t M[400];
    oracle_blosum62(M);
    for (int a = 0; a < 20; ++a)
        for (int b = 0; b < 20; ++b) out[20 * a + b] = (uint8_t)(a == b ? 0 : (M[20 * a + b] > 0 ? 1 : 2));
}

/* ------------------------------------------------------------------------- */
/* Per-pair gated fusion (Eq. alpha, Eq. wm, Eq. afused) with M = 2 channels:
 * a^(1) = s = S_ij / sqrt(S_ii S_jj) (normalised alignment, reading: geometric
 * mean of self-scores), a^(2) = c' = (1 + c)/2 with c the embedding cosine
 * (reading: shifted to [0,1]).  Channel scores are g^(1) = MLP(f), g^(2) = 0,
 * with f = [s, c, |L_i - L_j|] and MLP = w2 . ReLU(W1 f + b1) + b2, so Eq. wm
 * gives w^(1) = alpha = sigma(g) (Eq. alpha's sigmoid) and
 * fused = alpha s + (1 - alpha) c'.
 * params (float32, converted exactly): W1 [h][3] row-major, b1 [h], w2 [h], b2.
 * Pins: two-way softmax from a library routine, cosine from a library
 * routine, limits alpha -> 0 / 1, range [0, 1].                              */
/* ------------------------------------------------------------------------- */
typedef struct {
    double s, c, delta, alpha, g, fused, ni, nj;
} fuse_state;

static void fuse_pair(const uint32_t *pairs, int64_t p, const int32_t *sw, const int32_t *self,
                      const uint8_t *lens, const float *emb, int d, const float *params, int h,
                      double *z /* [h] */, fuse_state *st)
{
    uint32_t i = pairs[2 * p], j = pairs[2 * p + 1];
    const float *ei = emb + (int64_t)i * d, *ej = emb + (int64_t)j * d;
    double prod = (double)self[i] * (double)self[j];
    st->s = prod > 0.0 ? (double)sw[p] / sqrt(prod) : 0.0;
    double dot = 0.0, sii = 0.0, sjj = 0.0;
    for (int k = 0; k < d; ++k) {
        dot += (double)ei[k] * (double)ej[k];
        sii += (double)ei[k] * (double)ei[k];
        sjj += (double)ej[k] * (double)ej[k];
    }
    st->ni = sqrt(sii);
    st->nj = sqrt(sjj);
    st->c = (st->ni > 0.0 && st->nj > 0.0) ? dot / (st->ni * st->nj) : 0.0;
    st->delta = fabs((double)lens[i] - (double)lens[j]);
    const float *W1 = params, *b1 = params + 3 * h, *w2 = params + 4 * h, *b2 = params + 5 * h;
    double g = (double)b2[0];
    for (int k = 0; k < h; ++k) {
        z[k] = (double)W1[3 * k] * st->s + (double)W1[3 * k + 1] * st->c + (double)W1[3 * k + 2] * st->delta +
               (double)b1[k];
        g += (double)w2[k] * (z[k] > 0.0 ? z[k] : 0.0);
    }
    st->g = g;
    st->alpha = 1.0 / (1.0 + exp(-g));
    st->fused = st->alpha * st->s + (1.0 - st->alpha) * 0.5 * (1.0 + st->c);
}

int oracle_fuse_forward(const uint32_t *pairs, int64_t m, const int32_t *sw, const int32_t *self,
                        const uint8_t *lens, const float *emb, int d, const float *params, int h,
                        double *fused, double *alpha /* nullable */, double *snorm /* nullable */,
                        double *cosine /* nullable */)
{
    double *z = (double *)malloc((size_t)(h > 0 ? h : 1) * sizeof(double));
    if (!z) return -1;
    for (int64_t p = 0; p < m; ++p) {
        fuse_state st;
        fuse_pair(pairs, p, sw, self, lens, emb, d, params, h, z, &st);
        fused[p] = st.fused;
        if (alpha) alpha[p] = st.alpha;
        if (snorm) snorm[p] = st.s;
        if (cosine) cosine[p] = st.c;
    }
    free(z);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Adjoint of the fusion (gate training, Eq. fine_tune's meta-network
 * parameters).  Closed-form chain rule through fused, alpha, the MLP and the
 * cosine; the alignment channel is integer and not differentiated; the ReLU
 * subgradient at 0 is 0.  grad_params accumulates (caller zeroes); grad_emb
 * (nullable) accumulates dL/de_i and dL/de_j.
 * Pin: central finite differences of the forward + loss in a test.          */
/* ------------------------------------------------------------------------- */
int oracle_fuse_backward(const uint32_t *pairs, int64_t m, const int32_t *sw, const int32_t *self,
                         const uint8_t *lens, const float *emb, int d, const float *params, int h,
                         const double *dL_dfused, double *grad_params, double *grad_emb)
{
    double *z = (double *)malloc((size_t)(h > 0 ? h : 1) * sizeof(double));
    if (!z) return -1;
    const float *W1 = params, *w2 = params + 4 * h;
    double *gW1 = grad_params, *gb1 = grad_params + 3 * h, *gw2 = grad_params + 4 * h, *gb2 = grad_params + 5 * h;
    for (int64_t p = 0; p < m; ++p) {
        fuse_state st;
        fuse_pair(pairs, p, sw, self, lens, emb, d, params, h, z, &st);
        double dA = dL_dfused[p];
        double cprime = 0.5 * (1.0 + st.c);
        double d_alpha = dA * (st.s - cprime);
        double d_g = d_alpha * st.alpha * (1.0 - st.alpha);
        double d_c = dA * (1.0 - st.alpha) * 0.5;
        gb2[0] += d_g;
        for (int k = 0; k < h; ++k) {
            double u = z[k] > 0.0 ? z[k] : 0.0;
            gw2[k] += d_g * u;
            double d_z = z[k] > 0.0 ? d_g * (double)w2[k] : 0.0;
            gW1[3 * k] += d_z * st.s;
            gW1[3 * k + 1] += d_z * st.c;
            gW1[3 * k + 2] += d_z * st.delta;
            gb1[k] += d_z;
            d_c += d_z * (double)W1[3 * k + 1];
        }
        if (grad_emb && st.ni > 0.0 && st.nj > 0.0) {
            uint32_t i = pairs[2 * p], j = pairs[2 * p + 1];
            const float *ei = emb + (int64_t)i * d, *ej = emb + (int64_t)j * d;
            double inv = 1.0 / (st.ni * st.nj);
            for (int k = 0; k < d; ++k) {
                grad_emb[(int64_t)i * d + k] += d_c * ((double)ej[k] * inv - st.c * (double)ei[k] / (st.ni * st.ni));
                grad_emb[(int64_t)j * d + k] += d_c * ((double)ei[k] * inv - st.c * (double)ej[k] / (st.nj * st.nj));
            }
        }
    }
    free(z);
    return 0;
}

/* Rounding scale of the adjoint (no counterpart in the paper; used only to
 * state the FP32 tolerance of the GPU gradients).  For each parameter q,
 * scale[q] accumulates over pairs the contribution of pair p to
 * grad_params[q] evaluated on operand magnitudes, the quantity that bounds the
 * rounding error of a floating-point evaluation: every factor in absolute
 * value; a difference a - b by |a| + |b| (the channel difference s - c'); a
 * sum by the sum of its terms' magnitudes (the pre-activation z); the cosine
 * by 1 (its dot product's rounding error is relative to |e_i||e_j|); and the
 * ReLU taken as open for every pair (a pre-activation near zero may round to
 * either side).  scale_emb (nullable, [n][d]) does the same for grad_emb.  A
 * float32 evaluation of the chain differs from the exact gradient by at most
 * a small multiple of unit roundoff times this scale.  Both accumulate
 * (caller zeroes).                                                          */
int oracle_fuse_backward_scale(const uint32_t *pairs, int64_t m, const int32_t *sw, const int32_t *self,
                               const uint8_t *lens, const float *emb, int d, const float *params, int h,
                               const double *dL_dfused, double *scale, double *scale_emb)
{
    double *z = (double *)malloc((size_t)(h > 0 ? h : 1) * sizeof(double));
    if (!z) return -1;
    const float *W1 = params, *b1 = params + 3 * h, *w2 = params + 4 * h;
    double *sW1 = scale, *sb1 = scale + 3 * h, *sw2 = scale + 4 * h, *sb2 = scale + 5 * h;
    for (int64_t p = 0; p < m; ++p) {
        fuse_state st;
        fuse_pair(pairs, p, sw, self, lens, emb, d, params, h, z, &st);
        double dA = fabs(dL_dfused[p]);
        double diff = fabs(st.s) + 0.5 * (1.0 + fabs(st.c));
        double d_g = dA * diff * st.alpha * (1.0 - st.alpha);
        double d_c = dA * (1.0 - st.alpha) * 0.5;
        sb2[0] += d_g;
        for (int k = 0; k < h; ++k) {
            double zmag = fabs((double)W1[3 * k]) * st.s + fabs((double)W1[3 * k + 1]) +
                          fabs((double)W1[3 * k + 2]) * st.delta + fabs((double)b1[k]);
            sw2[k] += d_g * zmag;
            double d_z = d_g * fabs((double)w2[k]);
            sW1[3 * k] += d_z * st.s;
            sW1[3 * k + 1] += d_z;
            sW1[3 * k + 2] += d_z * st.delta;
            sb1[k] += d_z;
            d_c += d_z * fabs((double)W1[3 * k + 1]);
        }
        if (scale_emb && st.ni > 0.0 && st.nj > 0.0) {
            uint32_t i = pairs[2 * p], j = pairs[2 * p + 1];
            const float *ei = emb + (int64_t)i * d, *ej = emb + (int64_t)j * d;
            double inv = 1.0 / (st.ni * st.nj);
            for (int k = 0; k < d; ++k) {
                scale_emb[(int64_t)i * d + k] += d_c * (fabs((double)ej[k]) * inv + fabs((double)ei[k]) / (st.ni * st.ni));
                scale_emb[(int64_t)j * d + k] += d_c * (fabs((double)ei[k]) * inv + fabs((double)ej[k]) / (st.nj * st.nj));
            }
        }
    }
    free(z);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* M-channel gated fusion (Eq. wm with M > 2 channels, Eq. afused; Eq. alpha's
 * sigmoid is the M = 2 case).  Channels, in order:
 *   a^(1) = s  (normalised alignment, as above),
 *   a^(2) = c' = (1 + c)/2  (embedding cosine, as above),
 *   a^(3) = J  (MinHash estimate of the k-mer Jaccard index: the fraction of
 *               the H hash rows on which the two signatures agree; M = 3).
 * Reading: one two-layer MLP scores all channels from the features
 * f = [s, c, |L_i - L_j|, J] (J only for M = 3); its M - 1 outputs are the
 * logits of channels 1, 3, ..., and channel 2 keeps the fixed logit 0 (the
 * reference channel), so M = 2 is exactly the gate above.
 *   z = W1 f + b1 (h),  u = ReLU(z),  g^(1) = W2[0] . u + b2[0],  g^(2) = 0,
 *   g^(3) = W2[1] . u + b2[1];  w = softmax(g);  fused = sum_m w_m a^(m).
 * params (float32): W1 [h][F] row-major (F = M + 1), b1 [h], W2 [M-1][h]
 * row-major, b2 [M-1]; for M = 2 this is the layout of the two-channel gate.
 * sig: uint32 [n][H] sequence-major (the layout of oracle_sign).
 * Pins: softmax weights against a library softmax, weights sum to one,
 * M = 2 equals the two-channel gate, J against the exact agreement count,
 * channel limits (one dominant logit gives that channel's affinity).        */
/* ------------------------------------------------------------------------- */
typedef struct {
    double a[3], f[4], g[3], w[3], fused, c, ni, nj;
} mc_state;

static void fuse_pair_mc(const uint32_t *pairs, int64_t p, const int32_t *sw, const int32_t *self,
                         const uint8_t *lens, const float *emb, int d, const uint32_t *sig, int H, const float *params,
                         int h, int M, double *z /* [h] */, mc_state *st)
{
    uint32_t i = pairs[2 * p], j = pairs[2 * p + 1];
    const float *ei = emb + (int64_t)i * d, *ej = emb + (int64_t)j * d;
    double prod = (double)self[i] * (double)self[j];
    double s = prod > 0.0 ? (double)sw[p] / sqrt(prod) : 0.0;
    double dot = 0.0, sii = 0.0, sjj = 0.0;
    for (int k = 0; k < d; ++k) {
        dot += (double)ei[k] * (double)ej[k];
        sii += (double)ei[k] * (double)ei[k];
        sjj += (double)ej[k] * (double)ej[k];
    }
    st->ni = sqrt(sii);
    st->nj = sqrt(sjj);
    st->c = (st->ni > 0.0 && st->nj > 0.0) ? dot / (st->ni * st->nj) : 0.0;
    int F = M + 1;
    st->f[0] = s;
    st->f[1] = st->c;
    st->f[2] = fabs((double)lens[i] - (double)lens[j]);
    st->a[0] = s;
    st->a[1] = 0.5 * (1.0 + st->c);
    if (M == 3) {
        int agree = 0;
        for (int t = 0; t < H; ++t) agree += sig[(int64_t)i * H + t] == sig[(int64_t)j * H + t];
        st->a[2] = (double)agree / (double)H;
        st->f[3] = st->a[2];
    }
    const float *W1 = params, *b1 = params + F * h, *W2 = params + (F + 1) * h, *b2 = params + (F + M) * h;
    for (int k = 0; k < h; ++k) {
        double acc = (double)b1[k];
        for (int q = 0; q < F; ++q) acc += (double)W1[F * k + q] * st->f[q];
        z[k] = acc;
    }
    /* logits: channel 1 <- output 0, channel 2 <- 0, channel 3 <- output 1 */
    st->g[1] = 0.0;
    for (int r = 0; r < M - 1; ++r) {
        double acc = (double)b2[r];
        for (int k = 0; k < h; ++k) acc += (double)W2[r * h + k] * (z[k] > 0.0 ? z[k] : 0.0);
        st->g[r == 0 ? 0 : 2] = acc;
    }
    double mx = st->g[0];
    for (int q = 1; q < M; ++q)
        if (st->g[q] > mx) mx = st->g[q];
    double den = 0.0;
    for (int q = 0; q < M; ++q) den += exp(st->g[q] - mx);
    st->fused = 0.0;
    for (int q = 0; q < M; ++q) {
        st->w[q] = exp(st->g[q] - mx) / den;
        st->fused += st->w[q] * st->a[q];
    }
}

int oracle_fuse_forward_mc(const uint32_t *pairs, int64_t m, const int32_t *sw, const int32_t *self,
                           const uint8_t *lens, const float *emb, int d, const uint32_t *sig, int H,
                           const float *params, int h, int M, double *fused, double *weights /* [m][M], nullable */,
                           double *jacc /* [m], nullable */)
{
    if (M < 2 || M > 3 || (M == 3 && (!sig || H < 1))) return -2;
    double *z = (double *)malloc((size_t)(h > 0 ? h : 1) * sizeof(double));
    if (!z) return -1;
    for (int64_t p = 0; p < m; ++p) {
        mc_state st;
        fuse_pair_mc(pairs, p, sw, self, lens, emb, d, sig, H, params, h, M, z, &st);
        fused[p] = st.fused;
        if (weights)
            for (int q = 0; q < M; ++q) weights[p * M + q] = st.w[q];
        if (jacc) jacc[p] = M == 3 ? st.a[2] : 0.0;
    }
    free(z);
    return 0;
}

/* Adjoint of the M-channel fusion.  With fused = sum_m w_m a_m and w the
 * softmax of g, d fused / d g_k = w_k (a_k - fused); the logits' gradients
 * flow through W2, the ReLU (subgradient 0 at 0) and W1 to the parameters,
 * and with the channel c' = (1 + c)/2 and the feature c into the cosine and
 * the embeddings.  J is integer-derived and not differentiated.
 * grad_params (layout of params) and grad_emb (nullable, [n][d]) accumulate.
 * Pin: central finite differences of forward + loss in a test.              */
int oracle_fuse_backward_mc(const uint32_t *pairs, int64_t m, const int32_t *sw, const int32_t *self,
                            const uint8_t *lens, const float *emb, int d, const uint32_t *sig, int H,
                            const float *params, int h, int M, const double *dL_dfused, double *grad_params,
                            double *grad_emb)
{
    if (M < 2 || M > 3 || (M == 3 && (!sig || H < 1))) return -2;
    double *z = (double *)malloc((size_t)(h > 0 ? h : 1) * sizeof(double));
    if (!z) return -1;
    int F = M + 1;
    const float *W1 = params, *W2 = params + (F + 1) * h;
    double *gW1 = grad_params, *gb1 = grad_params + F * h, *gW2 = grad_params + (F + 1) * h,
           *gb2 = grad_params + (F + M) * h;
    for (int64_t p = 0; p < m; ++p) {
        mc_state st;
        fuse_pair_mc(pairs, p, sw, self, lens, emb, d, sig, H, params, h, M, z, &st);
        double dA = dL_dfused[p];
        double d_out[2]; /* gradient of MLP output r (logit of channel 1, then 3) */
        d_out[0] = dA * st.w[0] * (st.a[0] - st.fused);
        d_out[1] = M == 3 ? dA * st.w[2] * (st.a[2] - st.fused) : 0.0;
        double d_c = dA * st.w[1] * 0.5; /* through the channel c' */
        for (int r = 0; r < M - 1; ++r) gb2[r] += d_out[r];
        for (int k = 0; k < h; ++k) {
            double u = z[k] > 0.0 ? z[k] : 0.0;
            double du = 0.0;
            for (int r = 0; r < M - 1; ++r) {
                gW2[r * h + k] += d_out[r] * u;
                du += d_out[r] * (double)W2[r * h + k];
            }
            double d_z = z[k] > 0.0 ? du : 0.0;
            for (int q = 0; q < F; ++q) gW1[F * k + q] += d_z * st.f[q];
            gb1[k] += d_z;
            d_c += d_z * (double)W1[F * k + 1];
        }
        if (grad_emb && st.ni > 0.0 && st.nj > 0.0) {
            uint32_t i = pairs[2 * p], j = pairs[2 * p + 1];
            const float *ei = emb + (int64_t)i * d, *ej = emb + (int64_t)j * d;
            double inv = 1.0 / (st.ni * st.nj);
            for (int k = 0; k < d; ++k) {
                grad_emb[(int64_t)i * d + k] += d_c * ((double)ej[k] * inv - st.c * (double)ei[k] / (st.ni * st.ni));
                grad_emb[(int64_t)j * d + k] += d_c * ((double)ei[k] * inv - st.c * (double)ej[k] / (st.nj * st.nj));
            }
        }
    }
    free(z);
    return 0;
}

/* Rounding scale of the M-channel adjoint (test infrastructure, as
 * oracle_fuse_backward_scale): every pair's contribution evaluated on operand
 * magnitudes -- factors in absolute value, a difference a - b as |a| + |b|,
 * sums as the sum of their terms' magnitudes, the cosine as 1, the ReLU open.
 * scale (layout of params) and scale_emb (nullable) accumulate.             */
int oracle_fuse_backward_mc_scale(const uint32_t *pairs, int64_t m, const int32_t *sw, const int32_t *self,
                                  const uint8_t *lens, const float *emb, int d, const uint32_t *sig, int H,
                                  const float *params, int h, int M, const double *dL_dfused, double *scale,
                                  double *scale_emb)
{
    if (M < 2 || M > 3 || (M == 3 && (!sig || H < 1))) return -2;
    double *z = (double *)malloc((size_t)(h > 0 ? h : 1) * sizeof(double));
    if (!z) return -1;
    int F = M + 1;
    const float *W1 = params, *b1 = params + F * h, *W2 = params + (F + 1) * h;
    double *sW1 = scale, *sb1 = scale + F * h, *sW2 = scale + (F + 1) * h, *sb2 = scale + (F + M) * h;
    for (int64_t p = 0; p < m; ++p) {
        mc_state st;
        fuse_pair_mc(pairs, p, sw, self, lens, emb, d, sig, H, params, h, M, z, &st);
        double dA = fabs(dL_dfused[p]);
        double fmag[4] = {st.f[0], 1.0, st.f[2], M == 3 ? st.f[3] : 0.0};
        double amag = fabs(st.a[0]) + fabs(st.a[1]) + (M == 3 ? fabs(st.a[2]) : 0.0); /* bounds |fused| */
        double d_out[2];
        d_out[0] = dA * st.w[0] * (fabs(st.a[0]) + amag);
        d_out[1] = M == 3 ? dA * st.w[2] * (fabs(st.a[2]) + amag) : 0.0;
        double d_c = dA * st.w[1] * 0.5;
        for (int r = 0; r < M - 1; ++r) sb2[r] += d_out[r];
        for (int k = 0; k < h; ++k) {
            double zmag = fabs((double)b1[k]);
            for (int q = 0; q < F; ++q) zmag += fabs((double)W1[F * k + q]) * fmag[q];
            double du = 0.0;
            for (int r = 0; r < M - 1; ++r) {
                sW2[r * h + k] += d_out[r] * zmag;
                du += d_out[r] * fabs((double)W2[r * h + k]);
            }
            for (int q = 0; q < F; ++q) sW1[F * k + q] += du * fmag[q];
            sb1[k] += du;
            d_c += du * fabs((double)W1[F * k + 1]);
        }
        if (scale_emb && st.ni > 0.0 && st.nj > 0.0) {
            uint32_t i = pairs[2 * p], j = pairs[2 * p + 1];
            const float *ei = emb + (int64_t)i * d, *ej = emb + (int64_t)j * d;
            double inv = 1.0 / (st.ni * st.nj);
            for (int k = 0; k < d; ++k) {
                scale_emb[(int64_t)i * d + k] += d_c * (fabs((double)ej[k]) * inv + fabs((double)ei[k]) / (st.ni * st.ni));
                scale_emb[(int64_t)j * d + k] += d_c * (fabs((double)ei[k]) * inv + fabs((double)ej[k]) / (st.nj * st.nj));
            }
        }
    }
    free(z);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Training objective for the gate (reading: weighted binary cross-entropy of
 * the fused score against family-match labels; weight of a pair = inverse
 * frequency of its subgroup among the batch's pairs, normalised so the weights
 * sum to the number of pairs).  pair group g(p) = subgroup(i) if nonzero else
 * subgroup(j); label y_p = 1 iff i and j are in the same (non-background)
 * family.  p = clamp(fused, 1e-7, 1 - 1e-7).
 * Pins: torch's binary_cross_entropy with weights; the weights' sum.         */
/* ------------------------------------------------------------------------- */
void oracle_pair_labels(const uint32_t *pairs, int64_t m, const int32_t *family, const int32_t *subgroup,
                        uint8_t *label, int32_t *group)
{
    for (int64_t p = 0; p < m; ++p) {
        uint32_t i = pairs[2 * p], j = pairs[2 * p + 1];
        label[p] = (uint8_t)(family[i] >= 0 && family[i] == family[j]);
        group[p] = subgroup[i] != 0 ? subgroup[i] : subgroup[j];
    }
}

int oracle_pair_weights(const int32_t *group, int64_t m, int num_groups, double *weight)
{
    int64_t *count = (int64_t *)calloc((size_t)num_groups, sizeof(int64_t));
    if (!count) return -1;
    for (int64_t p = 0; p < m; ++p) {
        if (group[p] < 0 || group[p] >= num_groups) {
            free(count);
            return -1;
        }
        count[group[p]]++;
    }
    double total = 0.0;
    for (int64_t p = 0; p < m; ++p) total += (double)m / (double)count[group[p]]; /* 1 / pi_g */
    for (int64_t p = 0; p < m; ++p) weight[p] = ((double)m / (double)count[group[p]]) * (double)m / total;
    free(count);
    return 0;
}

#define BCE_EPS 1e-7

double oracle_bce_loss(const double *fused, const uint8_t *label, const double *weight, int64_t m,
                       double *dL_dfused /* nullable */)
{
    double wsum = 0.0, acc = 0.0;
    for (int64_t p = 0; p < m; ++p) wsum += weight[p];
    for (int64_t p = 0; p < m; ++p) {
        double q = fused[p];
        int inside = q > BCE_EPS && q < 1.0 - BCE_EPS;
        if (q < BCE_EPS) q = BCE_EPS;
        if (q > 1.0 - BCE_EPS) q = 1.0 - BCE_EPS;
        double y = (double)label[p];
        acc += weight[p] * -(y * log(q) + (1.0 - y) * log(1.0 - q));
        if (dL_dfused) dL_dfused[p] = inside ? weight[p] * (q - y) / (q * (1.0 - q)) / wsum : 0.0;
    }
    return acc / wsum;
}

/* Adam with bias correction (reading: beta1 0.9, beta2 0.999, eps 1e-8), one
 * step t >= 1 on P parameters.  Pin: torch.optim.Adam.                      */
void oracle_adam(double *param, const double *grad, double *m1, double *m2, int64_t P, int t, double lr,
                 double beta1, double beta2, double eps)
{
    double bc1 = 1.0 - pow(beta1, (double)t), bc2 = 1.0 - pow(beta2, (double)t);
    for (int64_t k = 0; k < P; ++k) {
        m1[k] = beta1 * m1[k] + (1.0 - beta1) * grad[k];
        m2[k] = beta2 * m2[k] + (1.0 - beta2) * grad[k] * grad[k];
        double mhat = m1[k] / bc1, vhat = m2[k] / bc2;
        param[k] -= lr * mhat / (sqrt(vhat) + eps);
    }
}

/* ------------------------------------------------------------------------- */
/* Cross-donor top-k retrieval over the candidate graph (recall@k is the
 * paper's retrieval quality measure).  For query q, the candidates are the
 * sequences j with {q, j} in C and donor(j) != donor(q); they are ranked by
 * (S(q,j) descending, j ascending) and the first k kept; unused slots are
 * id 0xffffffff, score -1.  Pin: brute force in a test.                      */
/* ------------------------------------------------------------------------- */
typedef struct {
    int32_t score;
    uint32_t id;
} scored_id;

static int cmp_scored(const void *pa, const void *pb)
{
    const scored_id *x = (const scored_id *)pa, *y = (const scored_id *)pb;
    if (x->score != y->score) return x->score > y->score ? -1 : 1;
    return (x->id > y->id) - (x->id < y->id);
}

int oracle_topk(const uint32_t *pairs, const int32_t *scores, int64_t m, const int32_t *donor,
                const uint32_t *queries, int64_t nq, int k, uint32_t *top_id, int32_t *top_score)
{
    scored_id *buf = NULL;
    int64_t cap = 0;
    for (int64_t qi = 0; qi < nq; ++qi) {
        uint32_t q = queries[qi];
        int64_t len = 0;
        for (int64_t p = 0; p < m; ++p) {
            uint32_t i = pairs[2 * p], j = pairs[2 * p + 1], other;
            if (i == q) other = j;
            else if (j == q) other = i;
            else continue;
            if (donor[other] == donor[q]) continue;
            if (len == cap) {
                int64_t nc = cap ? 2 * cap : 256;
                scored_id *nb = (scored_id *)realloc(buf, (size_t)nc * sizeof(scored_id));
                if (!nb) {
                    free(buf);
                    return -1;
                }
                buf = nb;
                cap = nc;
            }
            buf[len].score = scores[p];
            buf[len].id = other;
            ++len;
        }
        if (len > 0) qsort(buf, (size_t)len, sizeof(scored_id), cmp_scored);
        for (int r = 0; r < k; ++r) {
            top_id[qi * k + r] = r < len ? buf[r].id : 0xffffffffu;
            top_score[qi * k + r] = r < len ? buf[r].score : -1;
        }
    }
    free(buf);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Multi-threaded runners (the CPU baseline over all host cores; no new
 * arithmetic).  Each splits its index range into `threads` contiguous pieces
 * and calls the single-threaded routine above on each piece in its own POSIX
 * thread; results land in the same places, so the output is identical to the
 * single-threaded call.  Signatures are split by sequence, alignments and
 * fusion by pair; the candidate set by band (oracle_candidates_mt, after the
 * single-threaded per-band routine, with one final sort and deduplication). */
/* ------------------------------------------------------------------------- */
#include <pthread.h>

typedef struct {
    int kind; /* 0 sign, 1 sw, 2 fuse forward, 3 fuse backward (parameters only) */
    int64_t lo, hi;
    /* sign */
    const uint8_t *codes;
    int code_stride;
    const uint8_t *lens;
    int k, H;
    const uint32_t *a, *b;
    uint32_t *sig;
    /* sw */
    const uint32_t *pairs;
    const int32_t *M;
    int o, e;
    int32_t *scores;
    /* fuse */
    const int32_t *sw, *self;
    const float *emb, *params;
    int d, h;
    double *fused;
    const double *dL;
    double *grad; /* kind 3: this thread's own parameter-gradient partial */
    int rc;
} mt_job;

static void *mt_run(void *arg)
{
    mt_job *j = (mt_job *)arg;
    int64_t n = j->hi - j->lo;
    if (n <= 0) return NULL;
    if (j->kind == 0)
        oracle_sign(j->codes + j->lo * (int64_t)j->code_stride, j->code_stride, j->lens + j->lo, n, j->k, j->H, j->a,
                    j->b, j->sig + j->lo * (int64_t)j->H);
    else if (j->kind == 1)
        oracle_sw_pairs(j->codes, j->code_stride, j->lens, j->pairs + 2 * j->lo, n, j->M, j->o, j->e,
                        j->scores + j->lo);
    else if (j->kind == 2)
        j->rc = oracle_fuse_forward(j->pairs + 2 * j->lo, n, j->sw + j->lo, j->self, j->lens, j->emb, j->d, j->params,
                                    j->h, j->fused + j->lo, NULL, NULL, NULL);
    else
        j->rc = oracle_fuse_backward(j->pairs + 2 * j->lo, n, j->sw + j->lo, j->self, j->lens, j->emb, j->d, j->params,
                                     j->h, j->dL + j->lo, j->grad, NULL);
    return NULL;
}

static int mt_launch(mt_job *proto, int64_t count, int threads)
{
    if (threads < 1) threads = 1;
    if (threads > 1024) threads = 1024;
    mt_job *jobs = (mt_job *)calloc((size_t)threads, sizeof(mt_job));
    pthread_t *tid = (pthread_t *)calloc((size_t)threads, sizeof(pthread_t));
    int rc = 0;
    if (!jobs || !tid) {
        free(jobs);
        free(tid);
        return -1;
    }
    for (int t = 0; t < threads; ++t) {
        jobs[t] = *proto;
        jobs[t].lo = count * t / threads;
        jobs[t].hi = count * (t + 1) / threads;
        if (proto->kind == 3) jobs[t].grad = proto->grad + (int64_t)t * (5 * proto->h + 1);
        if (pthread_create(&tid[t], NULL, mt_run, &jobs[t]) != 0) {
            mt_run(&jobs[t]); /* run inline if a thread cannot be started */
            tid[t] = 0;
        }
    }
    for (int t = 0; t < threads; ++t) {
        if (tid[t]) pthread_join(tid[t], NULL);
        if (jobs[t].rc) rc = jobs[t].rc;
    }
    free(jobs);
    free(tid);
    return rc;
}

/* Candidates over `threads` threads: thread t runs band_chunk_pairs on its
 * own contiguous range of bands into its own vector (g_rows is set once
 * before the threads start); the vectors are concatenated, sorted and
 * deduplicated as in oracle_candidates, so the output is identical. */
typedef struct {
    const uint32_t *sig;
    int64_t n;
    int H, b0, b1, rows, cap, rc;
    u64vec part;
} cand_job;

static void *cand_run(void *arg)
{
    cand_job *j = (cand_job *)arg;
    if (j->b1 > j->b0)
        j->rc = band_chunk_pairs(j->sig + (int64_t)j->b0 * j->rows, j->n, j->H, j->b1 - j->b0, j->rows, j->cap,
                                 &j->part);
    return NULL;
}

int64_t oracle_candidates_mt(const uint32_t *sig, int64_t n, int H, int bands, int rows, int cap, uint32_t *out,
                             int64_t out_capacity, int threads)
{
    if (rows < 1 || rows > 8 || bands * rows > H) return -1;
    if (threads < 1) threads = 1;
    if (threads > bands) threads = bands;
    cand_job *jobs = (cand_job *)calloc((size_t)threads, sizeof(cand_job));
    pthread_t *tid = (pthread_t *)calloc((size_t)threads, sizeof(pthread_t));
    int rc = 0;
    if (!jobs || !tid) {
        free(jobs);
        free(tid);
        return -1;
    }
    g_rows = rows;
    for (int t = 0; t < threads; ++t) {
        jobs[t].sig = sig;
        jobs[t].n = n;
        jobs[t].H = H;
        jobs[t].rows = rows;
        jobs[t].cap = cap;
        jobs[t].b0 = (int)((int64_t)bands * t / threads);
        jobs[t].b1 = (int)((int64_t)bands * (t + 1) / threads);
        if (pthread_create(&tid[t], NULL, cand_run, &jobs[t]) != 0) {
            cand_run(&jobs[t]); /* run inline if a thread cannot be started */
            tid[t] = 0;
        }
    }
    int64_t total = 0;
    for (int t = 0; t < threads; ++t) {
        if (tid[t]) pthread_join(tid[t], NULL);
        if (jobs[t].rc) rc = jobs[t].rc;
        total += jobs[t].part.len;
    }
    u64vec all = {0, 0, 0};
    if (rc == 0 && total > 0) {
        all.v = (uint64_t *)malloc((size_t)total * sizeof(uint64_t));
        if (!all.v) rc = -1;
    }
    for (int t = 0; t < threads; ++t) {
        if (rc == 0 && jobs[t].part.len > 0) {
            memcpy(all.v + all.len, jobs[t].part.v, (size_t)jobs[t].part.len * sizeof(uint64_t));
            all.len += jobs[t].part.len;
        }
        free(jobs[t].part.v);
    }
    free(jobs);
    free(tid);
    if (rc != 0) {
        free(all.v);
        return -1;
    }
    all.cap = all.len;
    return sorted_unique_pairs(&all, out, out_capacity);
}

int oracle_sign_mt(const uint8_t *codes, int code_stride, const uint8_t *lens, int64_t n, int k, int H,
                   const uint32_t *a, const uint32_t *b, uint32_t *sig, int threads)
{
    mt_job j;
    memset(&j, 0, sizeof(j));
    j.kind = 0;
    j.codes = codes;
    j.code_stride = code_stride;
    j.lens = lens;
    j.k = k;
    j.H = H;
    j.a = a;
    j.b = b;
    j.sig = sig;
    return mt_launch(&j, n, threads);
}

int oracle_sw_pairs_mt(const uint8_t *codes, int code_stride, const uint8_t *lens, const uint32_t *pairs, int64_t m,
                       const int32_t *M, int o, int e, int32_t *scores, int threads)
{
    mt_job j;
    memset(&j, 0, sizeof(j));
    j.kind = 1;
    j.codes = codes;
    j.code_stride = code_stride;
    j.lens = lens;
    j.pairs = pairs;
    j.M = M;
    j.o = o;
    j.e = e;
    j.scores = scores;
    return mt_launch(&j, m, threads);
}

int oracle_fuse_forward_mt(const uint32_t *pairs, int64_t m, const int32_t *sw, const int32_t *self,
                           const uint8_t *lens, const float *emb, int d, const float *params, int h, double *fused,
                           int threads)
{
    mt_job j;
    memset(&j, 0, sizeof(j));
    j.kind = 2;
    j.pairs = pairs;
    j.sw = sw;
    j.self = self;
    j.lens = lens;
    j.emb = emb;
    j.d = d;
    j.params = params;
    j.h = h;
    j.fused = fused;
    return mt_launch(&j, m, threads);
}

/* Parameter gradient of the fusion adjoint over `threads` threads: thread t
 * accumulates its pair range into its own partial (the single-threaded
 * routine above); the partials are then added in thread order.  Summation
 * order differs from the single-threaded call (results agree to FP64
 * rounding).  grad_params accumulates (caller zeroes).                      */
int oracle_fuse_backward_params_mt(const uint32_t *pairs, int64_t m, const int32_t *sw, const int32_t *self,
                                   const uint8_t *lens, const float *emb, int d, const float *params, int h,
                                   const double *dL_dfused, double *grad_params, int threads)
{
    if (threads < 1) threads = 1;
    if (threads > 1024) threads = 1024;
    int P = 5 * h + 1;
    double *part = (double *)calloc((size_t)threads * (size_t)P, sizeof(double));
    if (!part) return -1;
    mt_job j;
    memset(&j, 0, sizeof(j));
    j.kind = 3;
    j.pairs = pairs;
    j.sw = sw;
    j.self = self;
    j.lens = lens;
    j.emb = emb;
    j.d = d;
    j.params = params;
    j.h = h;
    j.dL = dL_dfused;
    j.grad = part;
    int rc = mt_launch(&j, m, threads);
    for (int t = 0; t < threads; ++t)
        for (int q = 0; q < P; ++q) grad_params[q] += part[(int64_t)t * P + q];
    free(part);
    return rc;
}
