/*
 * hdc_oracle.c -- CPU oracle for the HDC classification path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this code; the product library never
 * does, and shares no code, header, table or helper with it.
 *
 * A plain, slow, obviously correct restatement, in FP64 / int64, of what the
 * GPU library computes.  Each function follows the paper "Compiler-Driven
 * Approximation Tuning for Hyperdimensional Computing" (ApproxHDC):
 *
 *   Sec. 2.1            encoding -> training by bundling -> inference by
 *                       similarity and nearest class
 *   Sec. 2.2, Listing 1 random-projection encoding (__hetero_hdc_matmul),
 *                       Hamming distance, red_perf(dists, 0.0, 0.5, 1) keeping
 *                       the first half of the dimensions, arg-min
 *   Sec. 4.2            Reduction Perforation (start, end, stride; similarity
 *                       results used unscaled), Automatic Binarization (+1/-1
 *                       stored as single bits, xor/popcount), Element Type
 *                       Representation (lower precision for inference),
 *                       Algorithmic Choice (cosine vs Hamming),
 *                       TRAIN_ITERATIONS (retraining epochs)
 *
 * Where the paper is silent the reading taken is stated at the function:
 * sign(0) = +1, lowest class index wins ties, perceptron retraining applied
 * once per epoch, power-of-two row scales for FP8, symmetric per-class
 * rounding for multi-bit class hypervectors.
 *
 * Binary hypervectors are held UNPACKED here, one byte per dimension, with
 * byte 1 meaning the element -1 and byte 0 meaning +1.
 *
 * Parity pins: every function is checked in the CPU test suite against
 * closed forms, invariants, library routines or brute force; none is
 * "parity unpinned".
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

/* ------------------------------------------------------------------------ */
/* Reduction perforation index set (Sec. 4.2 "Reduction Perforation";
 * Listing 1: red_perf(dists, 0.0, 0.5, 1) uses the first 1024 of 2048
 * elements, so start and end are fractions of D).
 * K = { s0 + k*stride : k >= 0, s0 + k*stride < e0 } with
 * s0 = floor(start*D), e0 = floor(end*D), both products formed in double.
 * Writes the kept dimensions to dims (if not NULL) and returns |K|,
 * or -1 when the arguments are out of range.                               */
int64_t orc_kept_dims(int64_t D, float start, float end, int64_t stride, int64_t *dims)
{
    if (D <= 0 || stride < 1 || !(start >= 0.0f) || !(end <= 1.0f) || !(start < end))
        return -1;
    int64_t s0 = (int64_t)floor((double)start * (double)D);
    int64_t e0 = (int64_t)floor((double)end * (double)D);
    int64_t n = 0;
    for (int64_t d = s0; d < e0; d += stride) {
        if (dims) dims[n] = d;
        n++;
    }
    return n;
}

/* Copy the columns listed in dims (Dk of them) of an n x D matrix.          */
void orc_gather_cols_u8(const uint8_t *src, int64_t n, int64_t D,
                        const int64_t *dims, int64_t Dk, uint8_t *dst)
{
    for (int64_t i = 0; i < n; i++)
        for (int64_t k = 0; k < Dk; k++)
            dst[i * Dk + k] = src[i * D + dims[k]];
}

void orc_gather_cols_i64(const int64_t *src, int64_t n, int64_t D,
                         const int64_t *dims, int64_t Dk, int64_t *dst)
{
    for (int64_t i = 0; i < n; i++)
        for (int64_t k = 0; k < Dk; k++)
            dst[i * Dk + k] = src[i * D + dims[k]];
}

/* ------------------------------------------------------------------------ */
/* Element types (Sec. 4.2 "Element Type Representation").
 *
 * BF16: 1 sign bit, 8 exponent bits (same range as FP32), 7 fraction bits.
 * Round to nearest, ties to even.  The spacing of representable values next
 * to |v| is 2^(e-7) with e = max(floor(log2|v|), -126).                     */
double orc_round_bf16(float v)
{
    double a = fabs((double)v);
    if (a == 0.0 || isinf(a) || isnan(a)) return (double)v;
    int ex;
    frexp(a, &ex);                 /* a = f * 2^ex, f in [0.5, 1) */
    int e = ex - 1;                /* floor(log2 a) */
    if (e < -126) e = -126;
    double ulp = ldexp(1.0, e - 7);
    double q = rint(a / ulp) * ulp; /* rint: current mode = nearest-even */
    return copysign(q, (double)v);
}

/* The same rounding of a double (no intermediate FP32 step): used for the
 * float query hypervectors, whose projections are formed in FP64 here.    */
double orc_round_bf16_f64(double v)
{
    double a = fabs(v);
    if (a == 0.0 || isinf(a) || isnan(a)) return v;
    int ex;
    frexp(a, &ex);
    int e = ex - 1;
    if (e < -126) e = -126;
    double ulp = ldexp(1.0, e - 7);
    double q = rint(a / ulp) * ulp;
    return copysign(q, v);
}

void orc_round_bf16_f64_array(const double *v, int64_t n, double *out)
{
    for (int64_t i = 0; i < n; i++) out[i] = orc_round_bf16_f64(v[i]);
}

/* FP8 E4M3 ("fn" variant: no infinities): 1 sign, 4 exponent bits with bias
 * 7, 3 fraction bits.  Normal values 2^e * (1 + m/8) for e in [-6, 8]; the
 * largest finite value is 448 = 2^8 * 1.75; subnormals are multiples of
 * 2^-9.  Round to nearest, ties to even, and clamp finite overflow to +-448
 * (the "satfinite" behaviour).                                             */
double orc_round_e4m3(double v)
{
    double a = fabs(v);
    if (a == 0.0 || isnan(a)) return v;
    int ex;
    frexp(a, &ex);
    int e = ex - 1;
    if (e < -6) e = -6;            /* subnormal range shares the 2^-9 spacing */
    double ulp = ldexp(1.0, e - 3);
    double q = rint(a / ulp) * ulp;
    if (q > 448.0) q = 448.0;
    return copysign(q, v);
}

/* Per-row power-of-two scale used with FP8 (our reading: the paper names
 * lower-precision types but no scaling rule).  The smallest s = 2^k with
 * amax <= 448 * s; s = 1 when amax = 0.                                     */
double orc_pow2_scale(double amax)
{
    if (!(amax > 0.0)) return 1.0;
    int k = ilogb(amax) - 8;
    while (amax > ldexp(448.0, k)) k++;
    while (amax <= ldexp(448.0, k - 1)) k--;
    return ldexp(1.0, k);
}

/* Quantise the rows of an n x F FP32 matrix for encoding type enc:
 *   0 = FP32 (unchanged), 1 = BF16, 2 = FP8 E4M3 with per-row scale.
 * out[i][f] holds the quantised value in units of scale[i]:
 *   x[i][f] ~= out[i][f] * scale[i].                                       */
void orc_quantise_rows(const float *x, int64_t n, int64_t F, int enc,
                       double *out, double *scale)
{
    for (int64_t i = 0; i < n; i++) {
        const float *r = x + i * F;
        double s = 1.0;
        if (enc == 2) {
            double amax = 0.0;
            for (int64_t f = 0; f < F; f++)
                if (fabs((double)r[f]) > amax) amax = fabs((double)r[f]);
            s = orc_pow2_scale(amax);
        }
        for (int64_t f = 0; f < F; f++) {
            double q;
            if (enc == 1)      q = orc_round_bf16(r[f]);
            else if (enc == 2) q = orc_round_e4m3((double)r[f] / s);
            else               q = (double)r[f];
            out[i * F + f] = q;
        }
        if (scale) scale[i] = s;
    }
}

/* ------------------------------------------------------------------------ */
/* Random-projection encoding (Sec. 2.1 encoding stage; Listing 1,
 * __hetero_hdc_matmul(input_features, rp_matrix) with rp_matrix stored as
 * D x F):  s[i][k] = sum_f x[i][f] * Bt[dims[k]][f], summed in f order.
 * FP64 version for real data, int64 version for integer data (exact).      */
void orc_encode_f64(const double *x, int64_t N, int64_t F, const double *Bt,
                    const int64_t *dims, int64_t Dk, double *s)
{
    for (int64_t i = 0; i < N; i++)
        for (int64_t k = 0; k < Dk; k++) {
            const double *b = Bt + dims[k] * F;
            double acc = 0.0;
            for (int64_t f = 0; f < F; f++) acc += x[i * F + f] * b[f];
            s[i * Dk + k] = acc;
        }
}

void orc_encode_i64(const int64_t *x, int64_t N, int64_t F, const int64_t *Bt,
                    const int64_t *dims, int64_t Dk, int64_t *s)
{
    for (int64_t i = 0; i < N; i++)
        for (int64_t k = 0; k < Dk; k++) {
            const int64_t *b = Bt + dims[k] * F;
            int64_t acc = 0;
            for (int64_t f = 0; f < F; f++) acc += x[i * F + f] * b[f];
            s[i * Dk + k] = acc;
        }
}

/* Absolute dot-product scale sum_f |x[i][f] * Bt[dims[k]][f]|, the size
 * against which the rounding error of a float encoding is measured.        */
void orc_encode_absdot_f64(const double *x, int64_t N, int64_t F, const double *Bt,
                           const int64_t *dims, int64_t Dk, double *s)
{
    for (int64_t i = 0; i < N; i++)
        for (int64_t k = 0; k < Dk; k++) {
            const double *b = Bt + dims[k] * F;
            double acc = 0.0;
            for (int64_t f = 0; f < F; f++) acc += fabs(x[i * F + f] * b[f]);
            s[i * Dk + k] = acc;
        }
}

/* Automatic Binarization (Sec. 4.2): map each element to +1 or -1; the
 * element -1 is stored as bit 1.  sign(0) = +1 (our reading), so bit = s < 0. */
void orc_binarise_f64(const double *s, int64_t n, uint8_t *bits)
{
    for (int64_t i = 0; i < n; i++) bits[i] = (s[i] < 0.0) ? 1 : 0;
}

void orc_binarise_i64(const int64_t *s, int64_t n, uint8_t *bits)
{
    for (int64_t i = 0; i < n; i++) bits[i] = (s[i] < 0) ? 1 : 0;
}

/* ------------------------------------------------------------------------ */
/* Hamming distance (Listing 1, __hetero_hdc_hamming_distance): the number of
 * positions in which two +-1 hypervectors differ, counted one position at a
 * time.  q is N x Dk, c is C x Dk (both already restricted to the kept
 * dimensions: a perforated reduction visits only those).  dist is N x C.    */
void orc_hamming(const uint8_t *q, int64_t N, const uint8_t *c, int64_t C,
                 int64_t Dk, int64_t *dist)
{
    for (int64_t i = 0; i < N; i++)
        for (int64_t j = 0; j < C; j++) {
            int64_t d = 0;
            for (int64_t k = 0; k < Dk; k++)
                if (q[i * Dk + k] != c[j * Dk + k]) d++;
            dist[i * C + j] = d;
        }
}

/* Arg-min (Listing 1, __hetero_hdc_arg_min): the nearest class; on a tie the
 * lowest class index wins (our reading).                                    */
void orc_argmin_i64(const int64_t *v, int64_t N, int64_t C, int32_t *label)
{
    for (int64_t i = 0; i < N; i++) {
        int64_t best = 0;
        for (int64_t j = 1; j < C; j++)
            if (v[i * C + j] < v[i * C + best]) best = j;
        label[i] = (int32_t)best;
    }
}

/* Arg-max for similarity scores; lowest index wins a tie.                  */
void orc_argmax_f64(const double *v, int64_t N, int64_t C, int32_t *label)
{
    for (int64_t i = 0; i < N; i++) {
        int64_t best = 0;
        for (int64_t j = 1; j < C; j++)
            if (v[i * C + j] > v[i * C + best]) best = j;
        label[i] = (int32_t)best;
    }
}

/* ------------------------------------------------------------------------ */
/* Class accumulators are int32 in the library; the oracle sums in int64 and
 * reports a result that int32 cannot hold.  Returns 1 when every entry lies
 * in [-2^31, 2^31 - 1], else 0.                                           */
int orc_acc_in_int32(const int64_t *acc, int64_t n)
{
    for (int64_t i = 0; i < n; i++)
        if (acc[i] < -2147483648LL || acc[i] > 2147483647LL) return 0;
    return 1;
}

/* Training by bundling (Sec. 2.1 training stage: same-class hypervectors are
 * added, then normalised).  acc[c][d] = sum over n with y_n = c of the +-1
 * element h[n][d] = 1 - 2*bit[n][d].  acc is overwritten.  Returns 0, or
 * -2 when an accumulator leaves the int32 range.                          */
int64_t orc_bundle(const uint8_t *bits, const int32_t *y, int64_t N, int64_t D,
                   int64_t C, int64_t *acc)
{
    for (int64_t i = 0; i < C * D; i++) acc[i] = 0;
    for (int64_t n = 0; n < N; n++) {
        int64_t c = y[n];
        if (c < 0 || c >= C) continue;
        for (int64_t d = 0; d < D; d++)
            acc[c * D + d] += 1 - 2 * (int64_t)bits[n * D + d];
    }
    return orc_acc_in_int32(acc, C * D) ? 0 : -2;
}

/* Normalisation of a bundled class hypervector = its sign (our reading of
 * "normalization" for binary models): class bit = acc < 0, sign(0) = +1.   */
void orc_class_bits(const int64_t *acc, int64_t C, int64_t D, uint8_t *cbits)
{
    for (int64_t i = 0; i < C * D; i++) cbits[i] = (acc[i] < 0) ? 1 : 0;
}

/* One retraining epoch (Sec. 4.2 TRAIN_ITERATIONS; the update rule is our
 * reading, the paper names only the epoch count).  Every sample is first
 * classified with the class bits taken from acc at the start of the epoch
 * (Hamming arg-min over all D dimensions); then, for each misclassified n,
 * acc[y_n] += h_n and acc[pred_n] -= h_n.  Returns the number of updates,
 * -1 when out of memory, or -2 when an accumulator leaves the int32 range
 * (acc then holds the int64 result).                                       */
int64_t orc_retrain_epoch(const uint8_t *bits, const int32_t *y, int64_t N,
                          int64_t D, int64_t C, int64_t *acc)
{
    uint8_t *cb = (uint8_t *)malloc((size_t)(C * D));
    int64_t *dist = (int64_t *)malloc(sizeof(int64_t) * (size_t)C);
    int32_t *pred = (int32_t *)malloc(sizeof(int32_t) * (size_t)(N > 0 ? N : 1));
    if (!cb || !dist || !pred) { free(cb); free(dist); free(pred); return -1; }
    orc_class_bits(acc, C, D, cb);
    for (int64_t n = 0; n < N; n++) {
        orc_hamming(bits + n * D, 1, cb, C, D, dist);
        orc_argmin_i64(dist, 1, C, pred + n);
    }
    int64_t updates = 0;
    for (int64_t n = 0; n < N; n++) {
        int64_t t = y[n], p = pred[n];
        if (t < 0 || t >= C || p == t) continue;
        for (int64_t d = 0; d < D; d++) {
            int64_t h = 1 - 2 * (int64_t)bits[n * D + d];
            acc[t * D + d] += h;
            acc[p * D + d] -= h;
        }
        updates++;
    }
    free(cb); free(dist); free(pred);
    return orc_acc_in_int32(acc, C * D) ? updates : -2;
}

/* ------------------------------------------------------------------------ */
/* b-bit class hypervectors (Sec. 4.2 "Element Type Representation": class
 * and query hypervectors projected onto lower-precision integers for
 * inference; the per-class symmetric rule is our reading).
 * b = 1: chat = +1 if acc >= 0 else -1.
 * b > 1: Q = 2^(b-1) - 1, M = max_d |acc[c][d]| over all D dimensions,
 *        chat = sign(acc) * floor((2|acc|Q + M) / (2M)), i.e. acc*Q/M rounded
 *        to the nearest integer with halves away from zero; M = 0 gives 0. */
void orc_class_quantise(const int64_t *acc, int64_t C, int64_t D, int b, int64_t *chat)
{
    for (int64_t c = 0; c < C; c++) {
        const int64_t *a = acc + c * D;
        int64_t *o = chat + c * D;
        if (b == 1) {
            for (int64_t d = 0; d < D; d++) o[d] = (a[d] >= 0) ? 1 : -1;
            continue;
        }
        int64_t Q = ((int64_t)1 << (b - 1)) - 1;
        int64_t M = 0;
        for (int64_t d = 0; d < D; d++) {
            int64_t m = a[d] < 0 ? -a[d] : a[d];
            if (m > M) M = m;
        }
        for (int64_t d = 0; d < D; d++) {
            if (M == 0) { o[d] = 0; continue; }
            int64_t m = a[d] < 0 ? -a[d] : a[d];
            int64_t r = (2 * m * Q + M) / (2 * M);
            o[d] = a[d] < 0 ? -r : r;
        }
    }
}

/* Cosine similarity (Sec. 4.2 "Algorithmic Choice": cosine instead of
 * Hamming) between the +-1 query q = 1 - 2*bit and each quantised class
 * hypervector, over the kept dimensions.  q is N x Dk, chat is C x Dk
 * (restricted to the same dimensions).  score = dot / sqrt(sum chat^2),
 * 0 when that norm is 0; the query norm sqrt(Dk) is the same for every class
 * and is left out.  dot and the squared norm are exact integers.           */
void orc_cosine_scores(const uint8_t *q, int64_t N, const int64_t *chat, int64_t C,
                       int64_t Dk, double *score)
{
    for (int64_t j = 0; j < C; j++) {
        int64_t nn = 0;
        for (int64_t k = 0; k < Dk; k++) nn += chat[j * Dk + k] * chat[j * Dk + k];
        double norm = sqrt((double)nn);
        for (int64_t i = 0; i < N; i++) {
            int64_t dot = 0;
            for (int64_t k = 0; k < Dk; k++)
                dot += (1 - 2 * (int64_t)q[i * Dk + k]) * chat[j * Dk + k];
            score[i * C + j] = (nn == 0) ? 0.0 : (double)dot / norm;
        }
    }
}

/* Cosine similarity of float query hypervectors (Sec. 4.2 Algorithmic
 * Choice: cosine on non-binarised hypervectors):
 *   score[i][j] = sum_k q[i][k] chat[j][k] / (||q_i|| ||chat_j||)
 * in FP64, 0 when either norm is 0.  q is N x Dk, chat is C x Dk.         */
void orc_cosine_float(const double *q, int64_t N, const int64_t *chat, int64_t C, int64_t Dk,
                      double *score)
{
    for (int64_t i = 0; i < N; i++) {
        double qq = 0.0;
        for (int64_t k = 0; k < Dk; k++) qq += q[i * Dk + k] * q[i * Dk + k];
        for (int64_t j = 0; j < C; j++) {
            double dot = 0.0, cc = 0.0;
            for (int64_t k = 0; k < Dk; k++) {
                dot += q[i * Dk + k] * (double)chat[j * Dk + k];
                cc += (double)chat[j * Dk + k] * (double)chat[j * Dk + k];
            }
            score[i * C + j] = (qq == 0.0 || cc == 0.0) ? 0.0 : dot / (sqrt(qq) * sqrt(cc));
        }
    }
}

/* Level-ID encoding (Sec. 4.2 Algorithmic Choice: ID-based encoding; the
 * Level-ID encoder of Micro-HD-Classification, Sec. 5.3).
 *
 * Quantisation of a feature to one of L levels over [x_lo, x_hi]:
 *   scale = (float)(L / (x_hi - x_lo))          (the quotient in double)
 *   t     = (x - lo) * scale                    (each operation in float)
 *   level = L-1 if t >= L, floor(t) if t > 0, else 0 (also for NaN).       */
float orc_levelid_scale(int32_t L, float x_lo, float x_hi)
{
    return (float)((double)L / ((double)x_hi - (double)x_lo));
}

void orc_levelid_quantise(const float *x, int64_t n, float lo, float scale, int32_t L, int32_t *level)
{
    for (int64_t i = 0; i < n; i++) {
        float d = x[i] - lo;
        float t = d * scale;
        if (t >= (float)L)
            level[i] = L - 1;
        else if (t > 0.0f)
            level[i] = (int32_t)floorf(t);
        else
            level[i] = 0;
    }
}

/* Level hypervectors: level l takes hi[d] where l >= flip[d], else lo[d]
 * (unpacked bits, 1 = element -1).                                        */
void orc_levelid_levels(const uint8_t *lo, const uint8_t *hi, const int32_t *flip, int64_t D, int32_t L,
                        uint8_t *levels)
{
    for (int32_t l = 0; l < L; l++)
        for (int64_t d = 0; d < D; d++) levels[(int64_t)l * D + d] = l >= flip[d] ? hi[d] : lo[d];
}

/* s[i][d] = sum_f id[f][d] * lev[level[i][f]][d] with bits mapped to +-1
 * (bit 1 = -1), exact in int64.                                            */
void orc_levelid_encode(const int32_t *level, int64_t N, int64_t F, const uint8_t *id, const uint8_t *lev,
                        int64_t D, int64_t *s)
{
    for (int64_t i = 0; i < N; i++)
        for (int64_t d = 0; d < D; d++) {
            int64_t acc = 0;
            for (int64_t f = 0; f < F; f++) {
                int64_t a = 1 - 2 * (int64_t)id[f * D + d];
                int64_t b = 1 - 2 * (int64_t)lev[(int64_t)level[i * F + f] * D + d];
                acc += a * b;
            }
            s[i * D + d] = acc;
        }
}
