/*
 * oracle.c -- plain, slow, single-threaded CPU statement of what the max_E SpMV
 * hot path computes (Jain et al., "Entropy Maximization in Sparse Matrix by
 * Vector Multiplication", arXiv 2308.00106).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path may link, load or call
 * this file: only the test suite, the smoke check and the benchmark's CPU
 * baseline do. It shares no code, header, table or constant generator with the
 * CUDA library; both sides implement the published definitions independently.
 *
 * Floating point is FP64 throughout. Stored values of the three value types are
 * decoded to double exactly (f32 and bf16 embed exactly in f64).
 *
 * Readings of the paper taken here (the paper leaves them open):
 *   - Permutation convention perm[new] = old, so A'[i',j'] = A[rperm[i'], cperm[j']],
 *     x'[j'] = x[cperm[j']], y[rperm[i']] = y'[i']  (Eq. 1, Section 1).
 *   - The pseudo-random permutation (Section 3; "Measuring", 32 seeded runs) is
 *     drawn by sorting 64-bit keys: key(seed, tag, i) is output number
 *     2*i + tag + 1 of the SplitMix64 generator seeded with `seed`
 *     (Steele, Lea, Flood, OOPSLA 2014; mixing constants of Stafford's Mix13).
 *     Ties in the key are broken by the index i.
 *   - CSR keeps columns ascending inside a row (Section 2), so a permuted row is
 *     re-sorted by its new column index (stable: equal columns keep their order).
 *   - Entropy (Section 4, Eq. "entropy") is taken over a gr x gc block grid of the
 *     matrix: bin(i, j) = (floor(i*gr/M), floor(j*gc/N)); H = -sum_{c>0} p log_b p,
 *     p = c / nnz, summed in row-major bin order. Base 2 by default.
 *   - SpMV (Section 2): y_i = sum over the stored row, in stored order.
 *   - Power iteration (used by the serving reference only; not in the paper):
 *     w = A v, v = w / ||w||_2, repeated; lambda = v^T A v.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { ORC_F64 = 0, ORC_F32 = 1, ORC_BF16 = 2 };

/* ---------------------------------------------------------------- values */

static double orc_decode(const void* val, int dtype, int64_t e) {
  if (dtype == ORC_F64) return ((const double*)val)[e];
  if (dtype == ORC_F32) return (double)((const float*)val)[e];
  /* bf16: the upper 16 bits of an IEEE binary32 */
  uint32_t bits = (uint32_t)((const uint16_t*)val)[e] << 16;
  float f;
  memcpy(&f, &bits, sizeof f);
  return (double)f;
}

static size_t orc_value_size(int dtype) {
  return dtype == ORC_F64 ? 8 : (dtype == ORC_F32 ? 4 : 2);
}

/* ------------------------------------------------ permutation (Section 3) */

/* SpMV-independent definition of SplitMix64: state advances by the golden
 * gamma 0x9e3779b97f4a7c15; output m (m >= 1) is mix(seed + m * gamma). */
uint64_t orc_key(uint64_t seed, int32_t tag, int64_t i) {
  uint64_t m = 2u * (uint64_t)i + (uint64_t)tag + 1u;
  uint64_t z = seed + m * 0x9e3779b97f4a7c15ULL;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

typedef struct {
  uint64_t key;
  int32_t idx;
} orc_pair;

static int orc_pair_cmp(const void* a, const void* b) {
  const orc_pair* p = (const orc_pair*)a;
  const orc_pair* q = (const orc_pair*)b;
  if (p->key != q->key) return p->key < q->key ? -1 : 1;
  return (p->idx > q->idx) - (p->idx < q->idx);
}

/* perm[new] = old: the indices 0..n-1 listed in ascending order of their keys. */
int orc_build_permutation(uint64_t seed, int32_t n, int32_t tag, int32_t* perm) {
  if (n < 0) return -1;
  orc_pair* pr = (orc_pair*)malloc(sizeof(orc_pair) * (size_t)(n > 0 ? n : 1));
  if (!pr) return -2;
  for (int32_t i = 0; i < n; ++i) {
    pr[i].key = orc_key(seed, tag, i);
    pr[i].idx = i;
  }
  qsort(pr, (size_t)n, sizeof(orc_pair), orc_pair_cmp);
  for (int32_t i = 0; i < n; ++i) perm[i] = pr[i].idx;
  free(pr);
  return 0;
}

/* inv[perm[i]] = i. Returns -1 if perm is not a bijection of 0..n-1. */
int orc_invert_permutation(const int32_t* perm, int32_t n, int32_t* inv) {
  for (int32_t i = 0; i < n; ++i) inv[i] = -1;
  for (int32_t i = 0; i < n; ++i) {
    int32_t p = perm[i];
    if (p < 0 || p >= n || inv[p] != -1) return -1;
    inv[p] = i;
  }
  return 0;
}

/* Vector forms of Eq. 1: x' = P_c^{-1} x is the gather out[i] = in[perm[i]];
 * y = P_r^{-1} y' is the scatter out[perm[i]] = in[i]. */
void orc_gather(const int32_t* perm, int32_t n, const double* in, double* out) {
  for (int32_t i = 0; i < n; ++i) out[i] = in[perm[i]];
}

void orc_scatter(const int32_t* perm, int32_t n, const double* in, double* out) {
  for (int32_t i = 0; i < n; ++i) out[perm[i]] = in[i];
}

/* --------------------------------------- permuted CSR (Section 1, Eq. 1) */

typedef struct {
  int32_t newcol;
  int32_t pos; /* position in the source row, keeps the sort stable */
  int64_t src; /* source index into col/val */
} orc_ent;

static int orc_ent_cmp(const void* a, const void* b) {
  const orc_ent* p = (const orc_ent*)a;
  const orc_ent* q = (const orc_ent*)b;
  if (p->newcol != q->newcol) return p->newcol < q->newcol ? -1 : 1;
  return (p->pos > q->pos) - (p->pos < q->pos);
}

/* A' = P_r A P_c: new row i' is old row rperm[i']; each old column c becomes
 * cinv[c]; the row is then sorted by new column. rperm / cperm may be NULL
 * (identity). Values are copied bit for bit. Returns 0, or -1 on a bad perm. */
int orc_permute_csr(int32_t M, int32_t N, const int32_t* rowptr, const int32_t* col,
                    const void* val, int dtype, const int32_t* rperm,
                    const int32_t* cperm, int32_t* rowptr_out, int32_t* col_out,
                    void* val_out) {
  size_t vs = orc_value_size(dtype);
  int32_t* cinv = (int32_t*)malloc(sizeof(int32_t) * (size_t)(N > 0 ? N : 1));
  if (!cinv) return -2;
  if (cperm) {
    if (orc_invert_permutation(cperm, N, cinv) != 0) {
      free(cinv);
      return -1;
    }
  } else {
    for (int32_t j = 0; j < N; ++j) cinv[j] = j;
  }
  int32_t maxlen = 0;
  for (int32_t i = 0; i < M; ++i) {
    int32_t len = rowptr[i + 1] - rowptr[i];
    if (len > maxlen) maxlen = len;
  }
  orc_ent* row = (orc_ent*)malloc(sizeof(orc_ent) * (size_t)(maxlen > 0 ? maxlen : 1));
  if (!row) {
    free(cinv);
    return -2;
  }
  int64_t out = 0;
  rowptr_out[0] = 0;
  for (int32_t ip = 0; ip < M; ++ip) {
    int32_t i = rperm ? rperm[ip] : ip;
    int32_t b = rowptr[i], e = rowptr[i + 1];
    for (int32_t t = b; t < e; ++t) {
      row[t - b].newcol = cinv[col[t]];
      row[t - b].pos = t - b;
      row[t - b].src = t;
    }
    qsort(row, (size_t)(e - b), sizeof(orc_ent), orc_ent_cmp);
    for (int32_t t = 0; t < e - b; ++t) {
      col_out[out] = row[t].newcol;
      memcpy((char*)val_out + (size_t)out * vs, (const char*)val + (size_t)row[t].src * vs, vs);
      ++out;
    }
    rowptr_out[ip + 1] = (int32_t)out;
  }
  free(row);
  free(cinv);
  return 0;
}

/* ---------------------------------------------- entropy (Section 4, Eq.) */

/* counts[br * gc + bc] = number of stored entries (i, j) with
 * floor(i*gr/M) = br and floor(j*gc/N) = bc.  Returns H in the given base
 * (H = 0 for an empty matrix). Requires 1 <= gr <= M and 1 <= gc <= N. */
double orc_nnz_entropy(int32_t M, int32_t N, const int32_t* rowptr, const int32_t* col,
                       int32_t gr, int32_t gc, double base, int64_t* counts) {
  int64_t nb = (int64_t)gr * gc;
  for (int64_t b = 0; b < nb; ++b) counts[b] = 0;
  for (int32_t i = 0; i < M; ++i) {
    int64_t br = (int64_t)i * gr / M;
    for (int32_t t = rowptr[i]; t < rowptr[i + 1]; ++t) {
      int64_t bc = (int64_t)col[t] * gc / N;
      counts[br * gc + bc] += 1;
    }
  }
  int64_t S = 0;
  for (int64_t b = 0; b < nb; ++b) S += counts[b];
  if (S == 0) return 0.0;
  double H = 0.0;
  for (int64_t b = 0; b < nb; ++b) {
    if (counts[b] == 0) continue; /* 0 log 0 = 0 */
    double p = (double)counts[b] / (double)S;
    double lg = (base == 2.0) ? log2(p) : log(p) / log(base);
    H -= p * lg;
  }
  return H;
}

/* Hierarchical 2-D entropy (Section 5: the entropy "split into 2x2, 4x4 and
 * 8x8"): the gr x gc count grid is cut into L x L blocks, block (a, b) taking
 * grid rows [ceil(a*gr/L), ceil((a+1)*gr/L)) and grid columns likewise; out[a*L+b]
 * is the entropy of the counts inside that block (0 for an empty block).
 * Requires 1 <= L <= gr, L <= gc. */
void orc_entropy_levels(const int64_t* counts, int32_t gr, int32_t gc, int32_t L, double base, double* out) {
  for (int32_t a = 0; a < L; ++a) {
    int64_t r0 = ((int64_t)a * gr + L - 1) / L, r1 = ((int64_t)(a + 1) * gr + L - 1) / L;
    for (int32_t b = 0; b < L; ++b) {
      int64_t c0 = ((int64_t)b * gc + L - 1) / L, c1 = ((int64_t)(b + 1) * gc + L - 1) / L;
      int64_t S = 0;
      for (int64_t i = r0; i < r1; ++i)
        for (int64_t j = c0; j < c1; ++j) S += counts[i * gc + j];
      double H = 0.0;
      if (S > 0) {
        for (int64_t i = r0; i < r1; ++i)
          for (int64_t j = c0; j < c1; ++j) {
            int64_t c = counts[i * gc + j];
            if (c == 0) continue;
            double p = (double)c / (double)S;
            H -= p * ((base == 2.0) ? log2(p) : log(p) / log(base));
          }
      }
      out[a * L + b] = H;
    }
  }
}

/* ---------------------------- gradient-based permutations (Section 5, appendix) */

/* Nonzero histogram along one axis: axis 0 gives the entries of each row
 * (M values), axis 1 the entries of each column (N values). */
void orc_nnz_histogram(int32_t M, int32_t N, const int32_t* rowptr, const int32_t* col, int32_t axis,
                       int32_t* hist) {
  if (axis == 0) {
    for (int32_t i = 0; i < M; ++i) hist[i] = rowptr[i + 1] - rowptr[i];
  } else {
    for (int32_t j = 0; j < N; ++j) hist[j] = 0;
    for (int64_t e = 0; e < (int64_t)rowptr[M]; ++e) hist[col[e]] += 1;
  }
}

/* Gradient-based permutation of n rows (or columns) from their histogram h.
 * Steps, in the paper's order:
 *   1. gradient g_i = h_{i+1} - h_i, i = 0..n-2;
 *   2. the pivot is the point of maximum steepness, max |g_i| (the first i on
 *      ties); the deck is cut before element i+1, so part one is [0, pivot) and
 *      part two [pivot, n), pivot = i+1 (pivot = n when n < 2: one part);
 *   3. riffle: cards are taken alternately from the top of part one and part
 *      two, starting with part one; when one part runs out the rest of the
 *      other follows in order;
 *   4. the shuffled deck is split into two parts again, its first ceil(n/2)
 *      cards and the rest, and each part is permuted at random: the positions
 *      q of a part are ordered by (key(seed, tag, q), q), the key of the
 *      Section 3 permutation.
 * perm[new] = old, as everywhere.  *pivot_out receives the cut (may be NULL). */
int orc_gradient_permutation(const int32_t* h, int32_t n, uint64_t seed, int32_t tag, int32_t* perm,
                             int32_t* pivot_out) {
  if (n < 0) return -1;
  int32_t pivot = n;
  if (n >= 2) {
    int64_t best = -1;
    for (int32_t i = 0; i + 1 < n; ++i) {
      int64_t g = (int64_t)h[i + 1] - (int64_t)h[i];
      int64_t steep = g < 0 ? -g : g;
      if (steep > best) {
        best = steep;
        pivot = i + 1;
      }
    }
  }
  if (pivot_out) *pivot_out = pivot;
  if (n == 0) return 0;
  int32_t* deck = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  orc_pair* pr = (orc_pair*)malloc(sizeof(orc_pair) * (size_t)n);
  if (!deck || !pr) {
    free(deck);
    free(pr);
    return -2;
  }
  /* 3. the riffle, card by card */
  int32_t top1 = 0, top2 = pivot, out = 0;
  int take_one = 1;
  while (out < n) {
    if (top1 < pivot && (take_one || top2 >= n)) {
      deck[out++] = top1++;
    } else {
      deck[out++] = top2++;
    }
    take_one = !take_one;
  }
  /* 4. random permutation inside each part of the shuffled deck */
  int32_t half = (n + 1) / 2;
  int32_t bounds[3] = {0, half, n};
  for (int part = 0; part < 2; ++part) {
    int32_t s = bounds[part], e = bounds[part + 1];
    for (int32_t q = s; q < e; ++q) {
      pr[q - s].key = orc_key(seed, tag, q);
      pr[q - s].idx = q;
    }
    qsort(pr, (size_t)(e - s), sizeof(orc_pair), orc_pair_cmp);
    for (int32_t t = 0; t < e - s; ++t) perm[s + t] = deck[pr[t].idx];
  }
  free(deck);
  free(pr);
  return 0;
}

/* ----------------------------------------------------- SpMV (Section 2) */

/* y_i = sum_{l in ROW[i]:ROW[i+1]} V[l] * x[COL[l]], in stored order, FP64. */
void orc_spmv(int32_t M, const int32_t* rowptr, const int32_t* col, const void* val,
              int dtype, const double* x, double* y) {
  for (int32_t i = 0; i < M; ++i) {
    double acc = 0.0;
    for (int32_t t = rowptr[i]; t < rowptr[i + 1]; ++t) acc += orc_decode(val, dtype, t) * x[col[t]];
    y[i] = acc;
  }
}

/* COO product (Section 2: triplets (ROW, COL, VALUE), no order required):
 * y = 0, then y[row[t]] += value[t] * x[col[t]] for t = 0..Z-1 in stored order. */
void orc_coo_spmv(int32_t M, int64_t Z, const int32_t* row, const int32_t* col, const void* val, int dtype,
                  const double* x, double* y) {
  for (int32_t i = 0; i < M; ++i) y[i] = 0.0;
  for (int64_t t = 0; t < Z; ++t) y[row[t]] += orc_decode(val, dtype, t) * x[col[t]];
}

/* Row indices of the COO form of a CSR matrix: row[t] = i for rowptr[i] <= t < rowptr[i+1]. */
void orc_csr_to_coo_rows(int32_t M, const int32_t* rowptr, int32_t* row) {
  for (int32_t i = 0; i < M; ++i)
    for (int32_t t = rowptr[i]; t < rowptr[i + 1]; ++t) row[t] = i;
}

/* Same product for k right-hand sides: X row-major N x k (leading dim ldx),
 * Y row-major M x k (leading dim ldy). */
void orc_spmm(int32_t M, const int32_t* rowptr, const int32_t* col, const void* val,
              int dtype, int32_t k, const double* X, int64_t ldx, double* Y, int64_t ldy) {
  for (int32_t i = 0; i < M; ++i) {
    for (int32_t c = 0; c < k; ++c) {
      double acc = 0.0;
      for (int32_t t = rowptr[i]; t < rowptr[i + 1]; ++t)
        acc += orc_decode(val, dtype, t) * X[(int64_t)col[t] * ldx + c];
      Y[(int64_t)i * ldy + c] = acc;
    }
  }
}

/* Exact rows only: y_i for a list of rows (used to check large cases one
 * output at a time). */
void orc_spmv_rows(const int32_t* rowptr, const int32_t* col, const void* val, int dtype,
                   const double* x, const int64_t* rows, int64_t nrows, double* y) {
  for (int64_t r = 0; r < nrows; ++r) {
    int64_t i = rows[r];
    double acc = 0.0;
    for (int32_t t = rowptr[i]; t < rowptr[i + 1]; ++t) acc += orc_decode(val, dtype, t) * x[col[t]];
    y[r] = acc;
  }
}

/* ------------------------------- power iteration (serving reference only) */

/* v <- A v / ||A v||_2 for `steps` steps starting at v0 (square A), then
 * lambda = v^T A v.  lam_hist[s] (if not NULL) receives the Rayleigh quotient
 * of the iterate after step s+1. Returns lambda; v_out receives v. */
double orc_power_iteration(int32_t M, const int32_t* rowptr, const int32_t* col,
                           const void* val, int dtype, const double* v0, int32_t steps,
                           double* v_out, double* lam_hist) {
  double* v = v_out;
  double* w = (double*)malloc(sizeof(double) * (size_t)(M > 0 ? M : 1));
  if (!w) return NAN;
  for (int32_t i = 0; i < M; ++i) v[i] = v0[i];
  double lam = 0.0;
  for (int32_t s = 0; s < steps; ++s) {
    orc_spmv(M, rowptr, col, val, dtype, v, w);
    double nrm = 0.0;
    for (int32_t i = 0; i < M; ++i) nrm += w[i] * w[i];
    nrm = sqrt(nrm);
    for (int32_t i = 0; i < M; ++i) v[i] = w[i] / nrm;
    if (lam_hist) {
      orc_spmv(M, rowptr, col, val, dtype, v, w);
      double d = 0.0;
      for (int32_t i = 0; i < M; ++i) d += v[i] * w[i];
      lam_hist[s] = d;
    }
  }
  orc_spmv(M, rowptr, col, val, dtype, v, w);
  for (int32_t i = 0; i < M; ++i) lam += v[i] * w[i];
  free(w);
  return lam;
}
