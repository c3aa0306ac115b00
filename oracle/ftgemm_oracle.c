/*
 * ftgemm_oracle.c -- CPU FP64 oracle for GEMM with online algorithm-based
 * fault tolerance (Wu, Zhai et al., "Anatomy of High-Performance GEMM with
 * Online Fault Tolerance on GPUs", ICS'23).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of bench.py load this library.  It shares no code, header or
 * table with the CUDA library; it is plain, slow and meant to be checked
 * against the paper by eye.
 *
 * What it computes
 *   (1) the plain definition C = alpha*A*B + beta*C_in in double precision
 *       (Section 3.1: the device-level problem C += A*B);
 *   (2) the ABFT algorithm step by step:
 *       - encoding: A^c = [A; e^T A] (Eq. 1), B^r = [B, B e] (Eq. 2);
 *       - full-checksum product C^f = A^c B^r holds C e and e^T C (Eq. 3);
 *       - outer-product form: the checksums are updated with every k-step s,
 *         C^f = sum_s A^c(:,s) B^r(s,:) (Eq. 4), so they stay valid in the
 *         middle of the computation and can be verified periodically;
 *       - verification against a threshold (Section 2.2), location by the
 *         flagged row and column, correction by subtracting the checksum
 *         offset (Section 4.2.1, "thread-level ABFT");
 *       - faults are additive offsets on accumulator values (Section 5.3);
 *       - single-event-upset model: one fault per unit and period (Section 4.1).
 *
 * Readings taken where the paper is silent (all listed in the design notes):
 *   - threshold, at a verification after k elements of K (of this split):
 *       tau^r_i = lambda*u*||A(i,:)||_2*||B(:,J_U)||_F + mu*u*sqrt(k)*|c^r_i|
 *       tau^c_j = lambda*u*||A(I_U,:)||_F*||B(:,j)||_2 + mu*u*sqrt(k)*|c^c_j|
 *     (norms over the full K; J_U/I_U are the columns/rows of the unit;
 *     c^r_i, c^c_j the checksums as they stand at the verification).  The
 *     first term is the size of the random-walk rounding error of zero-mean
 *     data; the second follows the growth of the partial sums of same-sign
 *     data, whose rounding error grows like u*sqrt(k) times the sum itself;
 *   - i* / j* = argmax |d|/tau, ties to the smallest index;
 *   - correction value = row residual d^r_{i*};  the pair is consistent only if
 *     |d^r_{i*} - d^c_{j*}| <= tau^r_{i*} + tau^c_{j*};
 *   - exactly one flagged row (or column) and no flagged column (row) means the
 *     checksum itself was hit: it is reset from the data and C is left alone;
 *   - any other flag pattern is uncorrectable (reported, C left alone);
 *   - the verification unit is the thread fragment, warp tile or block tile of
 *     the chosen level, with the fragment layout given by unit_row()/unit_col();
 *   - with split-K each split verifies its own partial sum; the sum of the
 *     splits and the alpha/beta epilogue are not protected;
 *   - detect-only (the offline scheme of Section 5.5): the unit is the whole
 *     tile and only its column checksums e^T C are compared, once per split
 *     (the schedule's cadence covers the split); a flagged column is reported
 *     as a detection (kind uncorrectable, no row) and nothing is corrected:
 *     the offline scheme recomputes the whole GEMM instead;
 *   - double precision (DGEMM, the extension named in Section 6) is (2) with
 *     u = 2^-53; double complex (ZGEMM) is (3): the same steps on complex
 *     values, one unit per output tile, |d| compared with a threshold built
 *     from the norms sqrt(sum |a|^2) and sqrt(sum |b|^2); a fault is a real
 *     or an imaginary offset.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* levels of the checksum unit (Section 4.2) */
enum { ORC_OFF = 0, ORC_THREAD = 1, ORC_WARP = 2, ORC_BLOCK = 3, ORC_TILE = 4, ORC_DETECT = 5 };
/* record kinds */
enum { ORC_CORRECTED = 0, ORC_UNCORRECTABLE = 1, ORC_CHECKSUM_ONLY = 2 };
/* fault targets */
enum { ORC_T_ACC = 0, ORC_T_ROWSUM = 1, ORC_T_COLSUM = 2 };

typedef struct {
  int32_t m_tb, n_tb, k_tb;   /* threadblock tile and k-step width (Table 1) */
  int32_t m_w, n_w, m_t, n_t; /* warp and thread tiles (Table 1) */
  int32_t cadence;            /* k-steps per verification period (>=1) */
  int32_t split_k;            /* number of K splits (>=1) */
  int32_t level;              /* ORC_* */
  double lambda;              /* threshold scale of the norm term */
  double u;                   /* unit roundoff of the accumulator */
  double mu;                  /* threshold scale of the checksum-growth term */
} orc_schedule;

typedef struct {
  int32_t tile_m, tile_n, kstep, row, col, target; /* row/col tile-local */
  double delta;
} orc_fault;

typedef struct {
  int32_t tile_m, tile_n, kstep, row, col, kind; /* row/col global, -1 if none */
  double delta, residual_r, residual_c, tau;
} orc_record;

/* ------------------------------------------------------------------------ */
/* (1) Plain definition: C = alpha * A B + beta * C_in, double precision     */
/*     (the problem of Section 3.1, with the scalars alpha and beta).        */
/* ------------------------------------------------------------------------ */
void orc_gemm_ref(int64_t M, int64_t N, int64_t K, double alpha,
                  const double* A, int64_t lda, const double* B, int64_t ldb,
                  double beta, const double* Cin, int64_t ldc, double* C,
                  int64_t ldo) {
  int64_t i;
#pragma omp parallel for schedule(static)
  for (i = 0; i < M; ++i) {
    for (int64_t j = 0; j < N; ++j) {
      double s = 0.0;
      for (int64_t k = 0; k < K; ++k) s += A[i * lda + k] * B[k * ldb + j];
      double c = alpha * s;
      if (beta != 0.0) c += beta * Cin[i * ldc + j];
      C[i * ldo + j] = c;
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Encoding (Eq. 1-2) per block of rows / columns, plus the norms used by   */
/* the threshold.  V[b][k] = sum_{i in row block b} A[i][k]                  */
/* W[b][k] = sum_{j in col block b} B[k][j]   (stored transposed: [b][k])    */
/* ------------------------------------------------------------------------ */
void orc_encode(int64_t M, int64_t N, int64_t K, const double* A, int64_t lda,
                const double* B, int64_t ldb, int32_t m_u, int32_t n_u,
                double* V, double* W, double* nA, double* nB) {
  int64_t mb = (M + m_u - 1) / m_u, nb = (N + n_u - 1) / n_u;
  for (int64_t b = 0; b < mb; ++b)
    for (int64_t k = 0; k < K; ++k) {
      double s = 0.0;
      for (int64_t i = b * m_u; i < M && i < (b + 1) * m_u; ++i) s += A[i * lda + k];
      V[b * K + k] = s;
    }
  for (int64_t b = 0; b < nb; ++b)
    for (int64_t k = 0; k < K; ++k) {
      double s = 0.0;
      for (int64_t j = b * n_u; j < N && j < (b + 1) * n_u; ++j) s += B[k * ldb + j];
      W[b * K + k] = s;
    }
  for (int64_t i = 0; i < M; ++i) {
    double s = 0.0;
    for (int64_t k = 0; k < K; ++k) s += A[i * lda + k] * A[i * lda + k];
    nA[i] = sqrt(s);
  }
  for (int64_t j = 0; j < N; ++j) {
    double s = 0.0;
    for (int64_t k = 0; k < K; ++k) s += B[k * ldb + j] * B[k * ldb + j];
    nB[j] = sqrt(s);
  }
}

/* ------------------------------------------------------------------------ */
/* Verification units.  A unit is (row group, column group) inside a tile.  */
/* Thread fragments follow the 4x8 lane layout of Table 1: a warp tile of    */
/* m_w x n_w has lm = m_w/m_t lanes along rows and ln = n_w/n_t along        */
/* columns; a thread's m_t rows come in chunks of vm = min(4, m_t)           */
/* consecutive rows, chunk c starting at c*lm*vm (columns likewise).         */
/* ------------------------------------------------------------------------ */
static int unit_row(const orc_schedule* s, int r) {
  switch (s->level) {
    case ORC_THREAD: {
      int lm = s->m_w / s->m_t, vm = s->m_t < 4 ? s->m_t : 4;
      int rw = r % s->m_w;
      int tm = (rw % (lm * vm)) / vm;
      return (r / s->m_w) * lm + tm;
    }
    case ORC_WARP: return r / s->m_w;
    default: return 0;
  }
}
static int unit_col(const orc_schedule* s, int c) {
  switch (s->level) {
    case ORC_THREAD: {
      int ln = s->n_w / s->n_t, vn = s->n_t < 4 ? s->n_t : 4;
      int cw = c % s->n_w;
      int tn = (cw % (ln * vn)) / vn;
      return (c / s->n_w) * ln + tn;
    }
    case ORC_WARP: return c / s->n_w;
    default: return 0;
  }
}
static int unit_rows(const orc_schedule* s) {
  switch (s->level) {
    case ORC_THREAD: return (s->m_tb / s->m_w) * (s->m_w / s->m_t);
    case ORC_WARP: return s->m_tb / s->m_w;
    default: return 1;
  }
}
static int unit_cols(const orc_schedule* s) {
  switch (s->level) {
    case ORC_THREAD: return (s->n_tb / s->n_w) * (s->n_w / s->n_t);
    case ORC_WARP: return s->n_tb / s->n_w;
    default: return 1;
  }
}

/* record list (per tile, merged at the end) */
typedef struct { orc_record* r; int32_t n, cap; } reclist;
static void rec_push(reclist* L, orc_record x) {
  if (L->n == L->cap) {
    L->cap = L->cap ? 2 * L->cap : 16;
    L->r = (orc_record*)realloc(L->r, sizeof(orc_record) * (size_t)L->cap);
  }
  L->r[L->n++] = x;
}
static int rec_cmp(const void* a, const void* b) {
  const orc_record* x = (const orc_record*)a;
  const orc_record* y = (const orc_record*)b;
  if (x->tile_m != y->tile_m) return x->tile_m < y->tile_m ? -1 : 1;
  if (x->tile_n != y->tile_n) return x->tile_n < y->tile_n ? -1 : 1;
  if (x->kstep != y->kstep) return x->kstep < y->kstep ? -1 : 1;
  if (x->row != y->row) return x->row < y->row ? -1 : 1;
  if (x->col != y->col) return x->col < y->col ? -1 : 1;
  return x->kind - y->kind;
}

static double score(double d, double tau) {
  double a = fabs(d);
  if (tau > 0.0) return a / tau;
  return a > 0.0 ? HUGE_VAL : 0.0;
}

/* ------------------------------------------------------------------------ */
/* (2) The ABFT algorithm: Eq. 1-2 per unit, the per-k-step update of Eq. 4, */
/*     verification and correction as in Section 4.2.1 at the unit of the   */
/*     level (Sections 4.2.1-4.2.3), faults as in Section 5.3, one fault    */
/*     per unit and period correctable (Section 4.1).                       */
/*   Cout[i*ldo+j] receives alpha*acc + beta*Cin.                            */
/*   counters[0..3] = detected, corrected, uncorrectable, checksum_only.     */
/*   Records are written sorted (tile_m, tile_n, kstep, row, col, kind);     */
/*   *nrec is the total count even if it exceeds cap.                       */
/*   Returns 0, or -1 on a bad argument.                                     */
/* ------------------------------------------------------------------------ */
int orc_gemm_ft(int64_t M, int64_t N, int64_t K, double alpha,
                const double* A, int64_t lda, const double* B, int64_t ldb,
                double beta, const double* Cin, int64_t ldc, double* Cout,
                int64_t ldo, const orc_schedule* sch, const orc_fault* faults,
                int32_t nfaults, orc_record* recs, int32_t cap,
                int64_t* counters, int32_t* nrec) {
  if (M <= 0 || N <= 0 || K <= 0 || !sch || sch->m_tb <= 0 || sch->n_tb <= 0 ||
      sch->k_tb <= 0 || sch->cadence <= 0 || sch->split_k <= 0)
    return -1;
  if (sch->level == ORC_THREAD &&
      (sch->m_w <= 0 || sch->n_w <= 0 || sch->m_t <= 0 || sch->n_t <= 0))
    return -1;
  if (sch->level == ORC_WARP && (sch->m_w <= 0 || sch->n_w <= 0)) return -1;

  const int mt = sch->m_tb, nt = sch->n_tb, kt = sch->k_tb;
  const int64_t tiles_m = (M + mt - 1) / mt, tiles_n = (N + nt - 1) / nt;
  const int64_t nks = (K + kt - 1) / kt;                  /* k-steps in total */
  const int64_t per_split = (nks + sch->split_k - 1) / sch->split_k;
  const int ngr = unit_rows(sch), ngc = unit_cols(sch);
  const int verify = sch->level != ORC_OFF;

  /* norms over the full K for the thresholds */
  double* nA = (double*)calloc((size_t)M, sizeof(double));
  double* nB = (double*)calloc((size_t)N, sizeof(double));
  for (int64_t i = 0; i < M; ++i) {
    double s = 0.0;
    for (int64_t k = 0; k < K; ++k) s += A[i * lda + k] * A[i * lda + k];
    nA[i] = sqrt(s);
  }
  for (int64_t j = 0; j < N; ++j) {
    double s = 0.0;
    for (int64_t k = 0; k < K; ++k) s += B[k * ldb + j] * B[k * ldb + j];
    nB[j] = sqrt(s);
  }

  int64_t cnt[4] = {0, 0, 0, 0};
  reclist all = {0, 0, 0};

  int64_t t;
#pragma omp parallel for schedule(dynamic, 1)
  for (t = 0; t < tiles_m * tiles_n; ++t) {
    const int64_t ti = t / tiles_n, tj = t % tiles_n;
    const int64_t i0 = ti * mt, j0 = tj * nt;
    const int rows = (int)(M - i0 < mt ? M - i0 : mt);
    const int cols = (int)(N - j0 < nt ? N - j0 : nt);
    double* acc = (double*)calloc((size_t)mt * nt, sizeof(double));
    double* cr = (double*)calloc((size_t)mt * ngc, sizeof(double)); /* row checksums */
    double* cc = (double*)calloc((size_t)nt * ngr, sizeof(double)); /* col checksums */
    double* dr = (double*)calloc((size_t)mt * ngc, sizeof(double));
    double* dc = (double*)calloc((size_t)nt * ngr, sizeof(double));
    double* tr = (double*)calloc((size_t)mt * ngc, sizeof(double));
    double* tc = (double*)calloc((size_t)nt * ngr, sizeof(double));
    double* er = (double*)calloc((size_t)mt * ngc, sizeof(double)); /* tau at this verification */
    double* ec = (double*)calloc((size_t)nt * ngr, sizeof(double));
    int64_t lc[4] = {0, 0, 0, 0};
    reclist L = {0, 0, 0};

    /* thresholds of every (row, column group) and (column, row group) */
    if (verify) {
      for (int g = 0; g < ngc; ++g) {
        double f = 0.0;
        for (int c = 0; c < cols; ++c)
          if (unit_col(sch, c) == g) f += nB[j0 + c] * nB[j0 + c];
        for (int r = 0; r < rows; ++r)
          tr[r * ngc + g] = sch->lambda * sch->u * nA[i0 + r] * sqrt(f);
      }
      for (int g = 0; g < ngr; ++g) {
        double f = 0.0;
        for (int r = 0; r < rows; ++r)
          if (unit_row(sch, r) == g) f += nA[i0 + r] * nA[i0 + r];
        for (int c = 0; c < cols; ++c)
          tc[c * ngr + g] = sch->lambda * sch->u * sqrt(f) * nB[j0 + c];
      }
    }

    for (int64_t sp = 0; sp < sch->split_k; ++sp) {
      const int64_t s0 = sp * per_split;
      const int64_t s1 = (s0 + per_split < nks) ? s0 + per_split : nks;
      if (s0 >= s1) continue;
      memset(acc, 0, sizeof(double) * (size_t)mt * nt);
      memset(cr, 0, sizeof(double) * (size_t)mt * ngc);
      memset(cc, 0, sizeof(double) * (size_t)nt * ngr);

      for (int64_t s = s0; s < s1; ++s) {
        const int64_t k0 = s * kt, k1 = (k0 + kt < K) ? k0 + kt : K;
        /* main accumulate: acc_IJ += A_I(:,s) B_J(s,:) */
        for (int r = 0; r < rows; ++r)
          for (int c = 0; c < cols; ++c) {
            double a = 0.0;
            for (int64_t k = k0; k < k1; ++k) a += A[(i0 + r) * lda + k] * B[k * ldb + j0 + c];
            acc[r * nt + c] += a;
          }
        if (verify) {
          /* row checksum  c^r += A_I(:,s) (B_J(s,:) e)   -- Eq. 2 and Eq. 4 */
          for (int g = 0; g < ngc; ++g)
            for (int64_t k = k0; k < k1; ++k) {
              double w = 0.0;
              for (int c = 0; c < cols; ++c)
                if (unit_col(sch, c) == g) w += B[k * ldb + j0 + c];
              for (int r = 0; r < rows; ++r) cr[r * ngc + g] += A[(i0 + r) * lda + k] * w;
            }
          /* column checksum  c^c += (e^T A_I(:,s)) B_J(s,:)   -- Eq. 1 and Eq. 4 */
          for (int g = 0; g < ngr; ++g)
            for (int64_t k = k0; k < k1; ++k) {
              double v = 0.0;
              for (int r = 0; r < rows; ++r)
                if (unit_row(sch, r) == g) v += A[(i0 + r) * lda + k];
              for (int c = 0; c < cols; ++c) cc[c * ngr + g] += v * B[k * ldb + j0 + c];
            }
        }
        /* faults scheduled after this k-step (Section 5.3) */
        for (int f = 0; f < nfaults; ++f) {
          const orc_fault* F = &faults[f];
          int64_t fk = F->kstep < 0 ? nks - 1 : F->kstep;
          if (F->tile_m != ti || F->tile_n != tj || fk != s) continue;
          if (F->row < 0 || F->row >= rows || F->col < 0 || F->col >= cols) continue;
          if (F->target == ORC_T_ROWSUM)
            cr[F->row * ngc + unit_col(sch, F->col)] += F->delta;
          else if (F->target == ORC_T_COLSUM)
            cc[F->col * ngr + unit_row(sch, F->row)] += F->delta;
          else
            acc[F->row * nt + F->col] += F->delta;
        }
        /* verification at the end of every period and at the split's end */
        const int64_t l = s - s0;
        if (!verify || !(((l + 1) % sch->cadence) == 0 || s == s1 - 1)) continue;
        /* thresholds at this verification: the norm term plus the growth term
           mu*u*sqrt(k)*|checksum|, k the elements of K accumulated so far */
        const double grow = sch->mu * sch->u * sqrt((double)(k1 - s0 * kt));
        for (int r = 0; r < rows; ++r)
          for (int g = 0; g < ngc; ++g) er[r * ngc + g] = tr[r * ngc + g] + grow * fabs(cr[r * ngc + g]);
        for (int c = 0; c < cols; ++c)
          for (int g = 0; g < ngr; ++g) ec[c * ngr + g] = tc[c * ngr + g] + grow * fabs(cc[c * ngr + g]);
        for (int gr = 0; gr < ngr; ++gr)
          for (int gc = 0; gc < ngc; ++gc) {
            int nr = 0, nc = 0, ib = -1, jb = -1;
            double sbr = -1.0, sbc = -1.0;
            for (int r = 0; r < rows && sch->level != ORC_DETECT; ++r) {
              if (unit_row(sch, r) != gr) continue;
              double S = 0.0;
              for (int c = 0; c < cols; ++c)
                if (unit_col(sch, c) == gc) S += acc[r * nt + c];
              double d = S - cr[r * ngc + gc];
              dr[r * ngc + gc] = d;
              double tau = er[r * ngc + gc];
              if (fabs(d) > tau) {
                ++nr;
                double sc = score(d, tau);
                if (sc > sbr) { sbr = sc; ib = r; }
              }
            }
            for (int c = 0; c < cols; ++c) {
              if (unit_col(sch, c) != gc) continue;
              double S = 0.0;
              for (int r = 0; r < rows; ++r)
                if (unit_row(sch, r) == gr) S += acc[r * nt + c];
              double d = S - cc[c * ngr + gr];
              dc[c * ngr + gr] = d;
              double tau = ec[c * ngr + gr];
              if (fabs(d) > tau) {
                ++nc;
                double sc = score(d, tau);
                if (sc > sbc) { sbc = sc; jb = c; }
              }
            }
            if (nr == 0 && nc == 0) continue;
            ++lc[0];
            if (sch->level == ORC_DETECT) {
              /* detect-only: report the most flagged column, correct nothing */
              orc_record rec;
              rec.tile_m = (int32_t)ti; rec.tile_n = (int32_t)tj; rec.kstep = (int32_t)s;
              rec.row = -1;
              rec.col = (int32_t)(j0 + jb);
              rec.residual_r = 0.0;
              rec.residual_c = dc[jb * ngr + gr];
              rec.tau = ec[jb * ngr + gr];
              rec.delta = 0.0;
              rec.kind = ORC_UNCORRECTABLE; ++lc[2];
              rec_push(&L, rec);
              continue;
            }
            orc_record rec;
            rec.tile_m = (int32_t)ti; rec.tile_n = (int32_t)tj; rec.kstep = (int32_t)s;
            rec.row = ib >= 0 ? (int32_t)(i0 + ib) : -1;
            rec.col = jb >= 0 ? (int32_t)(j0 + jb) : -1;
            rec.residual_r = ib >= 0 ? dr[ib * ngc + gc] : 0.0;
            rec.residual_c = jb >= 0 ? dc[jb * ngr + gr] : 0.0;
            rec.tau = (ib >= 0 ? er[ib * ngc + gc] : 0.0) + (jb >= 0 ? ec[jb * ngr + gr] : 0.0);
            rec.delta = 0.0;
            if (nr == 1 && nc == 1) {
              double drr = dr[ib * ngc + gc], dcc = dc[jb * ngr + gr];
              if (fabs(drr - dcc) <= er[ib * ngc + gc] + ec[jb * ngr + gr]) {
                acc[ib * nt + jb] -= drr; /* subtract the offset (Section 4.2.1) */
                rec.kind = ORC_CORRECTED; rec.delta = drr; ++lc[1];
              } else {
                rec.kind = ORC_UNCORRECTABLE; ++lc[2];
              }
            } else if ((nr == 1 && nc == 0) || (nr == 0 && nc == 1)) {
              /* a checksum was hit: reset it from the data, keep C */
              if (nr == 1) {
                double S = 0.0;
                for (int c = 0; c < cols; ++c)
                  if (unit_col(sch, c) == gc) S += acc[ib * nt + c];
                rec.delta = cr[ib * ngc + gc] - S;
                cr[ib * ngc + gc] = S;
              } else {
                double S = 0.0;
                for (int r = 0; r < rows; ++r)
                  if (unit_row(sch, r) == gr) S += acc[r * nt + jb];
                rec.delta = cc[jb * ngr + gr] - S;
                cc[jb * ngr + gr] = S;
              }
              rec.kind = ORC_CHECKSUM_ONLY; ++lc[3];
            } else {
              rec.kind = ORC_UNCORRECTABLE; ++lc[2];
            }
            rec_push(&L, rec);
          }
      }
      /* add this split's partial into Cout (the split sum is unprotected) */
      for (int r = 0; r < rows; ++r)
        for (int c = 0; c < cols; ++c) {
          if (sp == 0) Cout[(i0 + r) * ldo + j0 + c] = 0.0;
          Cout[(i0 + r) * ldo + j0 + c] += acc[r * nt + c];
        }
    }
    /* epilogue: C = alpha*acc + beta*C_in (unprotected) */
    for (int r = 0; r < rows; ++r)
      for (int c = 0; c < cols; ++c) {
        double v = alpha * Cout[(i0 + r) * ldo + j0 + c];
        if (beta != 0.0) v += beta * Cin[(i0 + r) * ldc + j0 + c];
        Cout[(i0 + r) * ldo + j0 + c] = v;
      }
#pragma omp critical
    {
      for (int q = 0; q < 4; ++q) cnt[q] += lc[q];
      for (int q = 0; q < L.n; ++q) rec_push(&all, L.r[q]);
    }
    free(L.r);
    free(acc); free(cr); free(cc); free(dr); free(dc); free(tr); free(tc); free(er); free(ec);
  }

  if (all.n > 1) qsort(all.r, (size_t)all.n, sizeof(orc_record), rec_cmp);
  for (int q = 0; q < all.n && q < cap; ++q) recs[q] = all.r[q];
  *nrec = all.n;
  for (int q = 0; q < 4; ++q) counters[q] = cnt[q];
  free(all.r);
  free(nA);
  free(nB);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* (3) Double-complex GEMM (ZGEMM), block-level units (Section 6 names DGEMM */
/* and ZGEMM as the extension of the scheme).  Matrices are interleaved      */
/* (re, im) pairs; leading dimensions count complex elements.                */
/* ------------------------------------------------------------------------ */
typedef struct {
  int32_t tile_m, tile_n, kstep, row, col, kind; /* row/col global, -1 if none */
  double delta_re, delta_im;                     /* amount subtracted / checksum offset */
  double res_r_re, res_r_im, res_c_re, res_c_im; /* residuals of the flagged row / column */
  double tau;
} orc_zrecord;

static double complex zat(const double* p, int64_t idx) { return p[2 * idx] + p[2 * idx + 1] * I; }

/* C = alpha * A B + beta * C_in, complex double precision (the plain        */
/* definition behind the ZGEMM extension of Section 6).                     */
void orc_zgemm_ref(int64_t M, int64_t N, int64_t K, const double* alpha,
                   const double* A, int64_t lda, const double* B, int64_t ldb,
                   const double* beta, const double* Cin, int64_t ldc, double* C,
                   int64_t ldo) {
  const double complex al = alpha[0] + alpha[1] * I, be = beta[0] + beta[1] * I;
  int64_t i;
#pragma omp parallel for schedule(static)
  for (i = 0; i < M; ++i) {
    for (int64_t j = 0; j < N; ++j) {
      double complex s = 0.0;
      for (int64_t k = 0; k < K; ++k) s += zat(A, i * lda + k) * zat(B, k * ldb + j);
      double complex c = al * s;
      if (be != 0.0) c += be * zat(Cin, i * ldc + j);
      C[2 * (i * ldo + j)] = creal(c);
      C[2 * (i * ldo + j) + 1] = cimag(c);
    }
  }
}

static int zrec_cmp(const void* a, const void* b) {
  const orc_zrecord* x = (const orc_zrecord*)a;
  const orc_zrecord* y = (const orc_zrecord*)b;
  if (x->tile_m != y->tile_m) return x->tile_m < y->tile_m ? -1 : 1;
  if (x->tile_n != y->tile_n) return x->tile_n < y->tile_n ? -1 : 1;
  if (x->kstep != y->kstep) return x->kstep < y->kstep ? -1 : 1;
  if (x->row != y->row) return x->row < y->row ? -1 : 1;
  if (x->col != y->col) return x->col < y->col ? -1 : 1;
  return x->kind - y->kind;
}

/* The online ABFT GEMM on complex values: tiles mt x nt, k-steps of kt,
 * verification every `cadence` k-steps and after the last (when verify).
 * Fault targets: low two bits as in (2); bit 2 set = the offset is imaginary
 * (delta * i).  Output and counters as in orc_gemm_ft. */
int orc_zgemm_ft(int64_t M, int64_t N, int64_t K, const double* alpha,
                 const double* A, int64_t lda, const double* B, int64_t ldb,
                 const double* beta, const double* Cin, int64_t ldc, double* Cout,
                 int64_t ldo, int32_t mt, int32_t nt, int32_t kt, int32_t cadence,
                 int32_t verify, double lambda, double u, double mu, const orc_fault* faults,
                 int32_t nfaults, orc_zrecord* recs, int32_t cap, int64_t* counters,
                 int32_t* nrec) {
  if (M <= 0 || N <= 0 || K <= 0 || mt <= 0 || nt <= 0 || kt <= 0 || cadence <= 0) return -1;
  const double complex al = alpha[0] + alpha[1] * I, be = beta[0] + beta[1] * I;
  const int64_t tiles_m = (M + mt - 1) / mt, tiles_n = (N + nt - 1) / nt;
  const int64_t nks = (K + kt - 1) / kt;

  /* norms over the full K: sqrt(sum |a|^2), sqrt(sum |b|^2) */
  double* nA = (double*)calloc((size_t)M, sizeof(double));
  double* nB = (double*)calloc((size_t)N, sizeof(double));
  for (int64_t i = 0; i < M; ++i) {
    double s = 0.0;
    for (int64_t k = 0; k < K; ++k) {
      double complex a = zat(A, i * lda + k);
      s += creal(a) * creal(a) + cimag(a) * cimag(a);
    }
    nA[i] = sqrt(s);
  }
  for (int64_t j = 0; j < N; ++j) {
    double s = 0.0;
    for (int64_t k = 0; k < K; ++k) {
      double complex b = zat(B, k * ldb + j);
      s += creal(b) * creal(b) + cimag(b) * cimag(b);
    }
    nB[j] = sqrt(s);
  }

  int64_t cnt[4] = {0, 0, 0, 0};
  orc_zrecord* all = NULL;
  int32_t nall = 0, capall = 0;

  int64_t t;
#pragma omp parallel for schedule(dynamic, 1)
  for (t = 0; t < tiles_m * tiles_n; ++t) {
    const int64_t ti = t / tiles_n, tj = t % tiles_n;
    const int64_t i0 = ti * mt, j0 = tj * nt;
    const int rows = (int)(M - i0 < mt ? M - i0 : mt);
    const int cols = (int)(N - j0 < nt ? N - j0 : nt);
    double complex* acc = (double complex*)calloc((size_t)mt * nt, sizeof(double complex));
    double complex* cr = (double complex*)calloc((size_t)mt, sizeof(double complex));
    double complex* cc = (double complex*)calloc((size_t)nt, sizeof(double complex));
    double complex* dr = (double complex*)calloc((size_t)mt, sizeof(double complex));
    double complex* dc = (double complex*)calloc((size_t)nt, sizeof(double complex));
    double* tr = (double*)calloc((size_t)mt, sizeof(double));
    double* tc = (double*)calloc((size_t)nt, sizeof(double));
    double* er = (double*)calloc((size_t)mt, sizeof(double)); /* tau at this verification */
    double* ec = (double*)calloc((size_t)nt, sizeof(double));
    orc_zrecord* L = NULL;
    int32_t nL = 0, capL = 0;
    int64_t lc[4] = {0, 0, 0, 0};

    /* thresholds: lambda*u*||A(i,:)||*||B(:,J)||_F and lambda*u*||A(I,:)||_F*||B(:,j)|| */
    double fa = 0.0, fb = 0.0;
    for (int r = 0; r < rows; ++r) fa += nA[i0 + r] * nA[i0 + r];
    for (int c = 0; c < cols; ++c) fb += nB[j0 + c] * nB[j0 + c];
    for (int r = 0; r < rows; ++r) tr[r] = lambda * u * nA[i0 + r] * sqrt(fb);
    for (int c = 0; c < cols; ++c) tc[c] = lambda * u * sqrt(fa) * nB[j0 + c];

    for (int64_t s = 0; s < nks; ++s) {
      const int64_t k0 = s * kt, k1 = (k0 + kt < K) ? k0 + kt : K;
      /* acc_IJ += A_I(:,s) B_J(s,:) */
      for (int r = 0; r < rows; ++r)
        for (int c = 0; c < cols; ++c) {
          double complex a = 0.0;
          for (int64_t k = k0; k < k1; ++k) a += zat(A, (i0 + r) * lda + k) * zat(B, k * ldb + j0 + c);
          acc[r * nt + c] += a;
        }
      if (verify) {
        for (int64_t k = k0; k < k1; ++k) {
          /* row checksum c^r += A_I(:,k) (B_J(k,:) e);  column checksum c^c += (e^T A_I(:,k)) B_J(k,:) */
          double complex w = 0.0, v = 0.0;
          for (int c = 0; c < cols; ++c) w += zat(B, k * ldb + j0 + c);
          for (int r = 0; r < rows; ++r) v += zat(A, (i0 + r) * lda + k);
          for (int r = 0; r < rows; ++r) cr[r] += zat(A, (i0 + r) * lda + k) * w;
          for (int c = 0; c < cols; ++c) cc[c] += v * zat(B, k * ldb + j0 + c);
        }
      }
      for (int f = 0; f < nfaults; ++f) {
        const orc_fault* F = &faults[f];
        int64_t fk = F->kstep < 0 ? nks - 1 : F->kstep;
        if (F->tile_m != ti || F->tile_n != tj || fk != s) continue;
        if (F->row < 0 || F->row >= rows || F->col < 0 || F->col >= cols) continue;
        const double complex off = (F->target & 4) ? F->delta * I : F->delta + 0.0 * I;
        switch (F->target & 3) {
          case ORC_T_ROWSUM: cr[F->row] += off; break;
          case ORC_T_COLSUM: cc[F->col] += off; break;
          default: acc[F->row * nt + F->col] += off; break;
        }
      }
      if (!verify || !(((s + 1) % cadence) == 0 || s == nks - 1)) continue;
      /* thresholds at this verification: the norm term plus the growth term
         mu*u*sqrt(k)*|checksum| after k elements of K */
      const double grow = mu * u * sqrt((double)k1);
      for (int r = 0; r < rows; ++r) er[r] = tr[r] + grow * cabs(cr[r]);
      for (int c = 0; c < cols; ++c) ec[c] = tc[c] + grow * cabs(cc[c]);
      int nr = 0, nc = 0, ib = -1, jb = -1;
      double sbr = -1.0, sbc = -1.0;
      for (int r = 0; r < rows; ++r) {
        double complex S = 0.0;
        for (int c = 0; c < cols; ++c) S += acc[r * nt + c];
        dr[r] = S - cr[r];
        if (cabs(dr[r]) > er[r]) {
          ++nr;
          double sc = score(cabs(dr[r]), er[r]);
          if (sc > sbr) { sbr = sc; ib = r; }
        }
      }
      for (int c = 0; c < cols; ++c) {
        double complex S = 0.0;
        for (int r = 0; r < rows; ++r) S += acc[r * nt + c];
        dc[c] = S - cc[c];
        if (cabs(dc[c]) > ec[c]) {
          ++nc;
          double sc = score(cabs(dc[c]), ec[c]);
          if (sc > sbc) { sbc = sc; jb = c; }
        }
      }
      if (nr == 0 && nc == 0) continue;
      ++lc[0];
      orc_zrecord rec;
      memset(&rec, 0, sizeof(rec));
      rec.tile_m = (int32_t)ti; rec.tile_n = (int32_t)tj; rec.kstep = (int32_t)s;
      rec.row = ib >= 0 ? (int32_t)(i0 + ib) : -1;
      rec.col = jb >= 0 ? (int32_t)(j0 + jb) : -1;
      if (ib >= 0) { rec.res_r_re = creal(dr[ib]); rec.res_r_im = cimag(dr[ib]); }
      if (jb >= 0) { rec.res_c_re = creal(dc[jb]); rec.res_c_im = cimag(dc[jb]); }
      rec.tau = (ib >= 0 ? er[ib] : 0.0) + (jb >= 0 ? ec[jb] : 0.0);
      double complex delta = 0.0;
      if (nr == 1 && nc == 1) {
        if (cabs(dr[ib] - dc[jb]) <= er[ib] + ec[jb]) {
          acc[ib * nt + jb] -= dr[ib]; /* subtract the offset (Section 4.2.1) */
          delta = dr[ib];
          rec.kind = ORC_CORRECTED; ++lc[1];
        } else {
          rec.kind = ORC_UNCORRECTABLE; ++lc[2];
        }
      } else if ((nr == 1 && nc == 0) || (nr == 0 && nc == 1)) {
        /* a checksum was hit: reset it from the data, keep C */
        if (nr == 1) {
          double complex S = 0.0;
          for (int c = 0; c < cols; ++c) S += acc[ib * nt + c];
          delta = cr[ib] - S;
          cr[ib] = S;
        } else {
          double complex S = 0.0;
          for (int r = 0; r < rows; ++r) S += acc[r * nt + jb];
          delta = cc[jb] - S;
          cc[jb] = S;
        }
        rec.kind = ORC_CHECKSUM_ONLY; ++lc[3];
      } else {
        rec.kind = ORC_UNCORRECTABLE; ++lc[2];
      }
      rec.delta_re = creal(delta);
      rec.delta_im = cimag(delta);
      if (nL == capL) {
        capL = capL ? 2 * capL : 16;
        L = (orc_zrecord*)realloc(L, sizeof(orc_zrecord) * (size_t)capL);
      }
      L[nL++] = rec;
    }
    /* epilogue: C = alpha*acc + beta*C_in (unprotected) */
    for (int r = 0; r < rows; ++r)
      for (int c = 0; c < cols; ++c) {
        double complex v = al * acc[r * nt + c];
        if (be != 0.0) v += be * zat(Cin, (i0 + r) * ldc + j0 + c);
        Cout[2 * ((i0 + r) * ldo + j0 + c)] = creal(v);
        Cout[2 * ((i0 + r) * ldo + j0 + c) + 1] = cimag(v);
      }
#pragma omp critical
    {
      for (int q = 0; q < 4; ++q) cnt[q] += lc[q];
      for (int q = 0; q < nL; ++q) {
        if (nall == capall) {
          capall = capall ? 2 * capall : 16;
          all = (orc_zrecord*)realloc(all, sizeof(orc_zrecord) * (size_t)capall);
        }
        all[nall++] = L[q];
      }
    }
    free(L);
    free(acc); free(cr); free(cc); free(dr); free(dc); free(tr); free(tc); free(er); free(ec);
  }

  if (nall > 1) qsort(all, (size_t)nall, sizeof(orc_zrecord), zrec_cmp);
  for (int q = 0; q < nall && q < cap; ++q) recs[q] = all[q];
  *nrec = nall;
  for (int q = 0; q < 4; ++q) counters[q] = cnt[q];
  free(all);
  free(nA);
  free(nB);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Low-precision inputs.  The ABFT checks run on the quantized values.       */
/* (No counterpart in the paper, whose kernels are fp32: these follow the   */
/* published bf16 and OCP FP8 formats.)                                     */
/* ------------------------------------------------------------------------ */

/* bfloat16: the top 16 bits of a binary32, rounded to nearest, ties to even */
void orc_round_bf16(const float* x, int64_t n, double* out) {
  for (int64_t i = 0; i < n; ++i) {
    float f = x[i];
    if (isnan(f)) { out[i] = (double)f; continue; }
    double a = fabs((double)f);
    if (a == 0.0 || isinf(f)) { out[i] = (double)f; continue; }
    /* bf16 keeps 8 significant bits: quantum = 2^(e-7) for a in [2^e, 2^(e+1)) */
    int e;
    frexp(a, &e);          /* a = m * 2^e, m in [0.5, 1) -> a in [2^(e-1), 2^e) */
    int ee = e - 1;
    if (ee < -126) ee = -126; /* subnormal range shares the smallest quantum */
    double q = ldexp(1.0, ee - 7);
    double r = nearbyint(a / q) * q; /* default rounding mode: ties to even */
    if (r > 3.3895313892515355e38) r = HUGE_VAL; /* overflow to inf */
    out[i] = f < 0 ? -r : r;
  }
}

/* OCP 8-bit floating point E4M3 (bias 7, max 448, no infinities):
 * x_q = sat(RNE(x / scale)); values returned already multiplied back by scale.
 * scale = amax(|x|) / 448 (1 if amax is 0).  The raw codes' values (before
 * the scale) are written to q_out if it is not NULL. */
double orc_quant_e4m3(const float* x, int64_t n, double* out, double* q_out) {
  double amax = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    double a = fabs((double)x[i]);
    if (a > amax) amax = a;
  }
  float scale = amax > 0.0 ? (float)amax / 448.0f : 1.0f;
  for (int64_t i = 0; i < n; ++i) {
    double v = (double)(x[i] / scale); /* fp32 division, as on the device */
    double a = fabs(v), r;
    if (a == 0.0) {
      r = 0.0;
    } else {
      int e;
      frexp(a, &e);
      int ee = e - 1;       /* a in [2^ee, 2^(ee+1)) */
      if (ee < -6) ee = -6; /* subnormals: quantum 2^-9 */
      double q = ldexp(1.0, ee - 3);
      r = nearbyint(a / q) * q;
      if (r > 448.0) r = 448.0; /* saturate */
    }
    r = v < 0 ? -r : r;
    if (q_out) q_out[i] = r;
    out[i] = r * (double)scale;
  }
  return (double)scale;
}

/* ------------------------------------------------------------------------ */
/* Online vs offline ABFT cost model (Section 5.5).                         */
/* gamma = 1 - (1 - gamma0)^(tiles); expected runs offline =                 */
/* (1 - gamma) / (1 - 2 gamma) for gamma < 1/2; online needs one run.        */
/* ------------------------------------------------------------------------ */
double orc_offline_expected_runs(double gamma0, double tiles) {
  double g = 1.0 - pow(1.0 - gamma0, tiles);
  if (g >= 0.5) return HUGE_VAL;
  return (1.0 - g) / (1.0 - 2.0 * g);
}

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
