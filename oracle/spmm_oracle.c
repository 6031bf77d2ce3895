/*
 * FP64 CPU oracle for the local CSR sparse-times-dense product.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or constant with the CUDA library: it is written from the
 * paper's definition of the operation and from the published number formats.
 *
 * What it computes (each function cites the passage it follows):
 *   oracle_spmm              C = beta*C0 + A*B, the local tile product
 *                            C_ij = C_ij + sum_k A_ik B_kj  (Section 2.1, the
 *                            stationary-C update, and Algorithm 2's
 *                            "local_c += local_a*local_b"), summed in FP64 over
 *                            the row's nonzeros in increasing CSR order.
 *   oracle_spmm_rows         the same for a list of rows (sampled checks).
 *   oracle_csr_transpose     CSR -> CSC (the CSR of A^T), stable in row order.
 *   oracle_sddmm             dv[e] = sum_n dC[row_e, n] * B[col_e, n].
 *   oracle_spmm_t_push       dB = A^T dC by scattering each nonzero's row of dC,
 *                            without forming the transpose.
 *   decode / encode          bfloat16, IEEE binary16 and OCP FP8 E4M3 from
 *                            their bit layouts; encoders round to nearest even,
 *                            E4M3 saturates to +-448.
 *   oracle_quantize_rows     per-row scaled E4M3: s = amax(row)/448 in FP32
 *                            (s = 1 for an all-zero row), q = E4M3(x / s).
 *   oracle_spgemm            the sparse-sparse local product C = A*B (the local
 *                            SpGEMM of Section 5's SpGEMM experiments): row i of
 *                            C holds column j when some k has A_ik and B_kj
 *                            stored (explicit zeros count), valued in FP64 as
 *                            sum_k A_ik B_kj; columns of each row increasing.
 *
 * The paper (Section 4) bounds the local product by the bytes of A, B and C;
 * the oracle makes no attempt at speed beyond an OpenMP loop over rows, which
 * leaves every row's summation order untouched.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_OK 0
#define ORACLE_ERR -1

void oracle_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int oracle_get_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* value readers: the dense and value arrays may be float32 or float64 */
static inline double rd(const void* p, int is_f32, int64_t i) {
    return is_f32 ? (double)((const float*)p)[i] : ((const double*)p)[i];
}

/* One output row of C = beta*C0 + A*B (Section 2.1): for each n, start from
 * beta*C0[r,n] (or 0 when beta == 0 or C0 is NULL), then add val_e*B[col_e,n]
 * for e = rowptr[r] .. rowptr[r+1]-1 in that order. */
static void spmm_one_row(int64_t r, int64_t N, const int32_t* rowptr, const int32_t* colind,
                         const void* vals, int vals_f32, const void* B, int b_f32, int64_t ldb,
                         double beta, const double* c0row, double* out) {
    for (int64_t n = 0; n < N; ++n)
        out[n] = (beta != 0.0 && c0row != NULL) ? beta * c0row[n] : 0.0;
    for (int64_t e = rowptr[r]; e < rowptr[r + 1]; ++e) {
        const double v = rd(vals, vals_f32, e);
        const int64_t k = colind[e];
        for (int64_t n = 0; n < N; ++n) out[n] += v * rd(B, b_f32, k * ldb + n);
    }
}

int oracle_spmm(int64_t M, int64_t K, int64_t N, const int32_t* rowptr, const int32_t* colind,
                const void* vals, int vals_f32, const void* B, int b_f32, int64_t ldb, double beta,
                const double* C0, int64_t ldc0, double* C, int64_t ldc) {
    (void)K;
    if (M < 0 || N < 0) return ORACLE_ERR;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t r = 0; r < M; ++r)
        spmm_one_row(r, N, rowptr, colind, vals, vals_f32, B, b_f32, ldb, beta,
                     C0 ? C0 + r * ldc0 : NULL, C + r * ldc);
    return ORACLE_OK;
}

/* Rows rows[0..nrows) of the same product, written densely to out[nrows x N].
 * C0rows (nullable) holds C0 at the sampled rows: row i of C0rows is C0[rows[i]]. */
int oracle_spmm_rows(int64_t N, const int32_t* rowptr, const int32_t* colind, const void* vals,
                     int vals_f32, const void* B, int b_f32, int64_t ldb, double beta,
                     const double* C0rows, int64_t ldc0, const int64_t* rows, int64_t nrows,
                     double* out) {
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < nrows; ++i)
        spmm_one_row(rows[i], N, rowptr, colind, vals, vals_f32, B, b_f32, ldb, beta,
                     C0rows ? C0rows + i * ldc0 : NULL, out + i * N);
    return ORACLE_OK;
}

/* CSR (M x K) -> CSC, i.e. the CSR of A^T (K x M).  Counting pass over the
 * column indices, exclusive prefix, then a scatter that walks rows in
 * increasing order, so every column lists its rows in increasing order.
 * perm[p] is the CSR position of the nonzero that lands at CSC position p. */
int oracle_csr_transpose(int64_t M, int64_t K, const int32_t* rowptr, const int32_t* colind,
                         const double* vals, int32_t* colptr, int32_t* rowind, double* tvals,
                         int64_t* perm) {
    int64_t* next = (int64_t*)calloc((size_t)K + 1, sizeof(int64_t));
    if (!next) return ORACLE_ERR;
    for (int64_t c = 0; c <= K; ++c) colptr[c] = 0;
    for (int64_t e = 0; e < rowptr[M]; ++e) {
        if (colind[e] < 0 || colind[e] >= K) { free(next); return ORACLE_ERR; }
        colptr[colind[e] + 1] += 1;
    }
    for (int64_t c = 0; c < K; ++c) colptr[c + 1] += colptr[c];
    for (int64_t c = 0; c < K; ++c) next[c] = colptr[c];
    for (int64_t r = 0; r < M; ++r) {
        for (int64_t e = rowptr[r]; e < rowptr[r + 1]; ++e) {
            const int64_t p = next[colind[e]]++;
            rowind[p] = (int32_t)r;
            if (tvals) tvals[p] = vals[e];
            if (perm) perm[p] = e;
        }
    }
    free(next);
    return ORACLE_OK;
}

/* Sampled dense-dense product at A's pattern: out[e] = sum_n dC[r,n]*B[col_e,n]
 * for every nonzero e of row r, n increasing, in FP64. */
int oracle_sddmm(int64_t M, int64_t N, const int32_t* rowptr, const int32_t* colind,
                 const void* dC, int dc_f32, int64_t lddc, const void* B, int b_f32, int64_t ldb,
                 double* out) {
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t r = 0; r < M; ++r) {
        for (int64_t e = rowptr[r]; e < rowptr[r + 1]; ++e) {
            const int64_t k = colind[e];
            double s = 0.0;
            for (int64_t n = 0; n < N; ++n)
                s += rd(dC, dc_f32, r * lddc + n) * rd(B, b_f32, k * ldb + n);
            out[e] = s;
        }
    }
    return ORACLE_OK;
}

/* dB = A^T dC without a transpose: dB = 0, then for every row r and every
 * nonzero e of r, dB[col_e, :] += val_e * dC[r, :].  Sequential, rows in
 * increasing order. */
int oracle_spmm_t_push(int64_t M, int64_t K, int64_t N, const int32_t* rowptr,
                       const int32_t* colind, const void* vals, int vals_f32, const void* dC,
                       int dc_f32, int64_t lddc, double* dB, int64_t lddb) {
    for (int64_t k = 0; k < K; ++k)
        for (int64_t n = 0; n < N; ++n) dB[k * lddb + n] = 0.0;
    for (int64_t r = 0; r < M; ++r) {
        for (int64_t e = rowptr[r]; e < rowptr[r + 1]; ++e) {
            const double v = rd(vals, vals_f32, e);
            const int64_t k = colind[e];
            for (int64_t n = 0; n < N; ++n) dB[k * lddb + n] += v * rd(dC, dc_f32, r * lddc + n);
        }
    }
    return ORACLE_OK;
}

/* ---------------- number formats ---------------- */

/* bfloat16: the upper 16 bits of an IEEE binary32. */
void oracle_decode_bf16(const uint16_t* in, int64_t n, double* out) {
    for (int64_t i = 0; i < n; ++i) {
        uint32_t bits = ((uint32_t)in[i]) << 16;
        float f;
        memcpy(&f, &bits, 4);
        out[i] = (double)f;
    }
}

/* IEEE binary16: 1 sign, 5 exponent (bias 15), 10 fraction bits. */
static double f16_value(uint16_t h) {
    const int s = (h >> 15) & 1, e = (h >> 10) & 0x1F, m = h & 0x3FF;
    double v;
    if (e == 0) v = ldexp((double)m, -24);
    else if (e == 31) v = (m == 0) ? INFINITY : NAN;
    else v = ldexp(1.0 + (double)m / 1024.0, e - 15);
    return s ? -v : v;
}

void oracle_decode_f16(const uint16_t* in, int64_t n, double* out) {
    for (int64_t i = 0; i < n; ++i) out[i] = f16_value(in[i]);
}

/* OCP FP8 E4M3 (the "fn" variant): 1 sign, 4 exponent (bias 7), 3 fraction
 * bits, no infinities, S.1111.111 is NaN, largest finite 1.75 * 2^8 = 448. */
static double e4m3_value(uint8_t q) {
    const int s = (q >> 7) & 1, e = (q >> 3) & 0xF, m = q & 0x7;
    double v;
    if (e == 0) v = ldexp((double)m, -9);
    else if (e == 15 && m == 7) v = NAN;
    else v = ldexp(1.0 + (double)m / 8.0, e - 7);
    return s ? -v : v;
}

void oracle_decode_e4m3(const uint8_t* in, int64_t n, double* out) {
    for (int64_t i = 0; i < n; ++i) out[i] = e4m3_value(in[i]);
}

/* Round-to-nearest-even of a non-negative double to an integer (the default
 * floating-point environment rounds half-way cases to even). */
static double rne(double x) { return nearbyint(x); }

/* float32 -> bfloat16, round to nearest even on the discarded 16 bits. */
void oracle_encode_bf16(const float* in, int64_t n, uint16_t* out) {
    for (int64_t i = 0; i < n; ++i) {
        uint32_t u;
        memcpy(&u, &in[i], 4);
        if ((u & 0x7F800000u) == 0x7F800000u && (u & 0x007FFFFFu)) {
            out[i] = (uint16_t)((u >> 16) | 0x0040u); /* quiet NaN */
            continue;
        }
        const uint32_t upper = u >> 16, lower = u & 0xFFFFu;
        uint32_t r = upper;
        if (lower > 0x8000u || (lower == 0x8000u && (upper & 1u))) r += 1; /* may carry to inf */
        out[i] = (uint16_t)r;
    }
}

/* float32 -> binary16, round to nearest even, overflow to infinity. */
void oracle_encode_f16(const float* in, int64_t n, uint16_t* out) {
    for (int64_t i = 0; i < n; ++i) {
        const double x = (double)in[i];
        uint16_t sign = signbit(x) ? 0x8000 : 0;
        const double a = fabs(x);
        uint16_t code;
        if (isnan(x)) { out[i] = 0x7E00; continue; }
        if (a >= 65520.0) code = 0x7C00;             /* half-way to 2^16 rounds up */
        else if (a < ldexp(1.0, -14)) {
            code = (uint16_t)rne(ldexp(a, 24));      /* 1024 = smallest normal */
        } else {
            int e;
            frexp(a, &e);                            /* a = f * 2^e, f in [0.5, 1) */
            e -= 1;                                  /* a = 1.xxx * 2^e */
            double m = rne((ldexp(a, -e) - 1.0) * 1024.0);
            if (m == 1024.0) { m = 0.0; e += 1; }
            code = (e + 15 >= 31) ? 0x7C00 : (uint16_t)(((e + 15) << 10) | (int)m);
        }
        out[i] = sign | code;
    }
}

/* float32 -> E4M3, round to nearest even, saturating finite values and
 * infinities to +-448; NaN -> 0x7F. */
static uint8_t e4m3_encode_one(float xf) {
    const double x = (double)xf;
    if (isnan(x)) return 0x7F;
    const uint8_t sign = signbit(x) ? 0x80 : 0;
    const double a = fabs(x);
    uint8_t code;
    if (a >= 448.0) code = 0x7E;
    else if (a < ldexp(1.0, -6)) {
        code = (uint8_t)rne(ldexp(a, 9));            /* 8 = smallest normal 2^-6 */
    } else {
        int e;
        frexp(a, &e);
        e -= 1;
        double m = rne((ldexp(a, -e) - 1.0) * 8.0);
        if (m == 8.0) { m = 0.0; e += 1; }
        code = (uint8_t)(((e + 7) << 3) | (int)m);
        if (code > 0x7E) code = 0x7E;
    }
    return sign | code;
}

void oracle_encode_e4m3(const float* in, int64_t n, uint8_t* out) {
    for (int64_t i = 0; i < n; ++i) out[i] = e4m3_encode_one(in[i]);
}

/* Per-row scaled E4M3: amax over the row in FP32, s = amax / 448 as an FP32
 * division (s = 1 when amax == 0), q = E4M3(x / s) with the quotient rounded to
 * FP32 first.  Dequantised value: decode(q) * s. */
void oracle_quantize_rows_e4m3(const float* X, int64_t rows, int64_t cols, int64_t ldx,
                               uint8_t* Q, int64_t ldq, float* scale) {
    for (int64_t r = 0; r < rows; ++r) {
        float amax = 0.0f;
        for (int64_t c = 0; c < cols; ++c) {
            const float a = fabsf(X[r * ldx + c]);
            if (a > amax) amax = a;
        }
        volatile float s = amax / 448.0f;
        if (amax == 0.0f) s = 1.0f;
        scale[r] = s;
        for (int64_t c = 0; c < cols; ++c) {
            volatile float q = X[r * ldx + c] / s;
            Q[r * ldq + c] = e4m3_encode_one(q);
        }
    }
}


/*
 * Local SpGEMM, C = A*B with A (M x K) and B (K x N) in CSR: a sparse
 * accumulator per row (a dense FP64 row of length N with a marker of the row
 * that last touched each column).  Call with C_colind == NULL to count: it
 * writes C_rowptr[M+1] only.  Then call again with C_colind and C_vals of
 * C_rowptr[M] entries to fill them.  Values are summed in FP64 over A's row in
 * CSR order and, within each term, over B's row in CSR order.
 */
static int cmp_i32(const void* a, const void* b) {
    const int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
    return (x > y) - (x < y);
}

int oracle_spgemm(int64_t M, int64_t K, int64_t N, const int32_t* A_rowptr,
                  const int32_t* A_colind, const double* A_vals, const int32_t* B_rowptr,
                  const int32_t* B_colind, const double* B_vals, int32_t* C_rowptr,
                  int32_t* C_colind, double* C_vals) {
    int64_t* mark = (int64_t*)malloc(sizeof(int64_t) * (size_t)(N > 0 ? N : 1));
    double* acc = (double*)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1));
    int32_t* cols = (int32_t*)malloc(sizeof(int32_t) * (size_t)(N > 0 ? N : 1));
    if (!mark || !acc || !cols) {
        free(mark); free(acc); free(cols);
        return ORACLE_ERR;
    }
    for (int64_t j = 0; j < N; ++j) mark[j] = -1;
    int64_t out = 0;
    if (!C_colind) C_rowptr[0] = 0;
    for (int64_t i = 0; i < M; ++i) {
        int64_t n = 0;
        for (int32_t e = A_rowptr[i]; e < A_rowptr[i + 1]; ++e) {
            const int32_t k = A_colind[e];
            if (k < 0 || k >= K) {
                free(mark); free(acc); free(cols);
                return ORACLE_ERR;
            }
            const double a = A_vals ? A_vals[e] : 1.0;
            for (int32_t f = B_rowptr[k]; f < B_rowptr[k + 1]; ++f) {
                const int32_t j = B_colind[f];
                if (j < 0 || j >= N) {
                    free(mark); free(acc); free(cols);
                    return ORACLE_ERR;
                }
                if (mark[j] != i) {
                    mark[j] = i;
                    acc[j] = 0.0;
                    cols[n++] = j;
                }
                acc[j] += a * (B_vals ? B_vals[f] : 1.0);
            }
        }
        if (!C_colind) {
            C_rowptr[i + 1] = (int32_t)(C_rowptr[i] + n);
            continue;
        }
        qsort(cols, (size_t)n, sizeof(int32_t), cmp_i32);
        for (int64_t q = 0; q < n; ++q) {
            C_colind[out + q] = cols[q];
            if (C_vals) C_vals[out + q] = acc[cols[q]];
        }
        out += n;
    }
    free(mark); free(acc); free(cols);
    return ORACLE_OK;
}
