// Internal declarations shared by the translation units of libhdc.
// Not part of the ABI (include/hdc.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "hdc.h"

namespace hdc {

constexpr int kAlign = 256;  // alignment of every sub-buffer we carve

// Training groups samples with int32 offsets over up to 2N entries (a
// retraining epoch places a misclassified sample in two groups) and 2C groups.
constexpr int64_t kMaxTrainRows = (int64_t(1) << 30) - 1;
constexpr int kMaxTrainClasses = 1 << 28;

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Words per packed row of L dims: ceil(L/32) rounded up to a multiple of 4.
inline int words_for(int64_t L) { return (int)((((L + 31) / 32) + 3) / 4 * 4); }

// Reduction-perforation index set (Sec. 4.2 "Reduction Perforation";
// Listing 1 red_perf(start, end, stride) with start/end fractions of D):
// kept dims are s0, s0+stride, ... below e0.
struct Perf {
    int64_t s0, e0, stride, Dk;
};
bool perf_of(int64_t D, const hdc_approx_config *cfg, Perf *p);

// Row stride of the quantised operands, in elements: a multiple of 128
// bytes, so every 128-byte TMA box row is one aligned L2 line (a 16-byte
// stride measured 1.6x slower in the tensor-core kernel); the zero padding
// costs 14% more bytes at F = 784, which the compute-bound kernel hides.
// 32 floats for the FP32 copy of the base.
inline int ld_for(int enc, int F) {
    int q = enc == HDC_ENC_BF16 ? 64 : enc == HDC_ENC_FP8_E4M3 ? 128 : 32;
    return (F + q - 1) / q * q;
}
inline int esize_for(int enc) { return enc == HDC_ENC_BF16 ? 2 : enc == HDC_ENC_FP8_E4M3 ? 1 : 4; }

// ---- launchers (each returns the launch error) -----------------------------

// K1: quantise rows src[row_off + k*row_step] (F floats each, row stride lds)
// into dst row k (ldd elements, zero padded); FP8 writes the row's power-of-
// two scale to scale[k].  enc: HDC_ENC_FP32 (copy), BF16, FP8_E4M3.  With
// (c0, cstep) != (0, 1), element f of a row is source column c0 + f*cstep
// (the kept features of a perforated encoding reduction).
cudaError_t launch_quant_rows(const float *src, int64_t lds, int64_t row_off, int64_t row_step,
                              int64_t nrows, int F, int enc, void *dst, int ldd, float *scale,
                              cudaStream_t st, int64_t c0 = 0, int64_t cstep = 1);

// Class preparation: planes [b][C][W] (or, with vals, the b-bit values as
// BF16 rows of ldv elements, zero past Dk), sums and norms over the kept dims.
cudaError_t launch_class_prepare(const int32_t *acc, int C, int D, const Perf &p, int b,
                                 uint32_t *planes, int W, int32_t *csum, double *cnorm,
                                 uint16_t *vals, int ldv, cudaStream_t st);

// Binary class planes (C x W words) -> E4M3 +-1 bytes (Cp x ldcs; 0 past Dk
// and for rows C..Cp-1) for the tensor-core Hamming distances.
cudaError_t launch_class_sign(const uint32_t *planes, int C, int W, int Dk, int Cp, int ldcs, uint8_t *out,
                              cudaStream_t st);

// FP32 projections (N x Dk, from the CUDA-core encoder) -> BF16 rows of ldS
// elements (zero past Dk) and the squared norms of the BF16 rows.
cudaError_t launch_proj_bf16(const float *s, int64_t N, int Dk, uint16_t *q, int ldS, float *qn,
                             cudaStream_t st);

// K0: CUDA-core encode + sign + pack: H (N x W), optional scores (N x Dk).
// X: N x ldx elements of type enc (FP32 rows may be unpadded: ldx = F),
// Bq: Dk x ldb elements of type enc.  sx / sb: row scales or NULL.
cudaError_t launch_encode_simt(const void *X, int64_t ldx, int64_t N, int F, const void *Bq, int ldb,
                               int Dk, int enc, const float *sx, const float *sb, uint32_t *H, int W,
                               float *scores, cudaStream_t st);

// K4: similarity + arg-min/arg-max over packed hypervectors.
//  nb == 1: Hamming distance to plane 0, masked by perforation p over D
//           (p == NULL: every dim of W words counts), arg-min.
//  nb  > 1: cosine score from nb two's-complement planes, arg-max.
cudaError_t launch_similarity(const uint32_t *Q, int64_t N, const uint32_t *planes, int C, int W,
                              int nb, int64_t D, const Perf *p, const int32_t *csum,
                              const double *cnorm, int32_t *labels, int32_t *dists, double *scores,
                              cudaStream_t st);

// Hamming arg-min of N packed rows H against C <= 16 binary classes over all
// W words (pred), counting the retraining groups of each misclassified row
// into hist (2C int32, zeroed by the caller): hist[y]++ and hist[C + pred]++.
// cudaErrorNotSupported for C > 16.
cudaError_t launch_argmin_groups(const uint32_t *H, int64_t N, const uint32_t *cls, int C, int W, const int32_t *y,
                                 int32_t *pred, int32_t *hist, cudaStream_t st);

// K5: one training pass over N packed rows H (W words, D dims, C classes):
//  mode 0: acc = per-class sums of (1 - 2 bit) (bundling), cls_out = sign;
//  mode 1: pred = Hamming arg-min against cls_in; rows with pred != y add to
//          y and subtract from pred: acc += that, cls_out = sign(acc);
//  mode 2: as mode 1, but acc = the updates alone and cls_out is NULL.
// n_updates (if not NULL, zeroed by the caller) counts the updated rows.
// Scratch (train_max_items(N, C) counting items): perm (2N int32), hist and
// cursor (2C int32), offsets and items (2C + 1 int32), partial (max items x
// W x 8 uint32 byte lanes).
// signs: for 33..256 classes, Cp x hamming_packed_ldcs(W) bytes for the
// class hypervectors expanded once per epoch (NULL: the Hamming kernel
// expands them itself).
struct TrainScratch {
    int32_t *perm, *hist, *offsets, *items, *cursor;
    uint32_t *partial;
    uint8_t *signs;
};
// Bytes of the expanded class hypervectors the training and clustering
// workspaces hold (0 outside 33..256 classes).
size_t class_sign_bytes(int C, int W);
// Hamming arg-min of N packed rows against C classes over the kept dims
// (s0, s0 + stride, ... < e0; all of [0, D) for a stride-1 full range): the
// library's routes, with the class hypervectors expanded into `signs`
// (class_sign_bytes(C, W), or NULL) for the tensor-core route.
cudaError_t launch_argmin_ws(const uint32_t *H, int64_t N, const uint32_t *cls, int C, int W, int64_t D,
                             const Perf *p, int32_t *labels, uint8_t *signs, cudaStream_t st);
int64_t train_max_items(int64_t N, int C);
cudaError_t launch_train_pass(const uint32_t *H, int W, const int32_t *y, int64_t N, int D, int C, int mode,
                              const uint32_t *cls_in, int32_t *pred, int32_t *acc, uint32_t *cls_out,
                              int32_t *n_updates, const TrainScratch &s, cudaStream_t st);

// K6 (binary): cls[c] = pack(acc[c] < 0) over D dims, W words per row.
cudaError_t launch_binarise(const int32_t *acc, int C, int D, uint32_t *cls, int W, cudaStream_t st);
// K6 with the exchange step of sharded training: acc += delta (delta may be
// NULL), then cls = pack(acc < 0).
cudaError_t launch_apply_binarise(const int32_t *delta, int32_t *acc, int C, int D, uint32_t *cls, int W,
                                  cudaStream_t st);

// Tensor-core (tcgen05) encode, fused with Hamming / cosine and arg-min.
// Returns cudaErrorNotSupported when the shape is outside what it handles.
struct TcArgs {
    const void *Xq;   // N x ldx quantised queries (BF16 or FP8)
    int64_t N;
    int F;            // features (the contraction length)
    int ldx;          // elements per row (16-byte multiple, >= F)
    const void *Bq;   // Dk x ldb quantised base rows
    int ldb;
    int Dk;
    int enc;
    const float *sx, *sb;       // row scales (FP8) or NULL
    uint32_t *H;                // encode-only output (N x W) or NULL
    float *scores;              // optional N x Dk projections
    uint16_t *sproj;            // encode-only: BF16 projections (N x ldS) or NULL
    int ldS;
    float *qn;                  // with sproj: squared norms of the BF16 rows
    const uint8_t *cls_sign;    // classify, binary classes: E4M3 +-1 class bytes (Cp x ldcs) or NULL
    int ldcs;
    int W;
    // fused similarity (classify); planes == NULL for encode-only
    const uint32_t *planes;
    int C, nb;
    const int32_t *csum;
    const double *cnorm;
    int32_t *labels, *dists;
    double *sims;
    // classify only: the FP32 query rows (N x ldX) to quantise inside the
    // kernel, with `stage` (tc_stage_bytes) for its staged query tiles;
    // Xq is then unused
    const float *X;
    int64_t ldX;
    uint8_t *stage;
    // classify (binary classes, the popcount epilogue): scratch of
    // tc_split_bytes(N, C) zero-filled per launch, so that a batch of few
    // query tiles can split each tile's dim tiles over several CTAs; NULL
    // keeps one CTA per query tile
    int32_t *dacc;
};
// Query tiles whose dim tiles a fused classify may split over CTAs, and the
// scratch that needs: partial distances of those tiles' rows (int32 x C) and
// one counter per tile.
constexpr int64_t TC_SPLIT_MAX_TILES = 256;
inline size_t tc_split_bytes(int64_t N, int C)
{
    const int64_t rows = N < TC_SPLIT_MAX_TILES * 128 ? N : TC_SPLIT_MAX_TILES * 128;
    return (size_t)rows * C * 4 + (size_t)TC_SPLIT_MAX_TILES * 4;
}
cudaError_t launch_tc_encode(const TcArgs &a, cudaStream_t st);
bool tc_supported(const TcArgs &a);
// Whether the fused classify of a can quantise its own query tiles from the
// FP32 rows a.X (binary classes: up to 32, or up to 112 with their E4M3
// signs; 16-byte aligned rows of F % 4 == 0 floats; ldx <= 1024; at least two
// tiles per CTA; at least 0.15 * F 128-byte MMA stages per query tile, below
// which the row-quantiser pass is faster), and the bytes its staged tiles
// take (at most N rows of the quantised operand).
bool tc_qin_ok(const TcArgs &a);
size_t tc_stage_bytes(const TcArgs &a);

// Reads and clears the streaming quantiser's device status word.
cudaError_t quant_read_status(cudaStream_t st, int *status);

// Reads and clears the tensor-core kernels' device status word.
cudaError_t tc_read_status(cudaStream_t st, int *status);
// Hamming arg-min of packed rows on the tensor cores (17 <= C <= 256 binary
// classes, W a multiple of 4 up to 4096): kept dims s0 + k*stride < min(e0, D).
bool hamming_packed_ok(int C, int W);
// cls_sign (optional): the class hypervectors already expanded by
// launch_class_sign(cls, C, W, Dk, Cp, hamming_packed_ldcs(W), cls_sign) --
// the kernel then streams them instead of expanding the class words itself.
int hamming_packed_ldcs(int W);
cudaError_t launch_hamming_packed(const uint32_t *Q, int64_t N, const uint32_t *cls, int C, int W, int64_t D,
                                  int64_t s0, int64_t e0, int64_t stride, int32_t *labels, int32_t *dists,
                                  cudaStream_t st, const uint8_t *cls_sign = nullptr);
// One block waiting, bounded by limit_ns, on a barrier nothing arrives on
// (the expiry is reported through tc_read_status).
cudaError_t launch_wait_selftest(unsigned long long limit_ns, cudaStream_t st);

// Cosine of float query hypervectors on the tensor cores (k_tc_cos.cu):
// q (N x ldS BF16), qn (N squared norms), cv (Cp x ldS BF16 class values,
// Cp = C rounded up to 16, C <= 256), cnorm (C) -> labels, optional scores.
struct CosArgs {
    const uint16_t *q;
    const float *qn;
    int64_t N;
    int ldS;
    const uint16_t *cv;
    const double *cnorm;
    int C, Cp;
    int32_t *labels;
    double *scores;
};
cudaError_t launch_tc_cosine(const CosArgs &a, cudaStream_t st);

// Float queries with C <= 112 classes, encode and cosine fused (tc_fcos.cuh):
// the encoder operands of `a` (Xq, Bq, scales, Dk, C, labels), the BF16 class
// values cv (Cp x ldS) and their norms; cudaErrorNotSupported outside it.
cudaError_t launch_tc_fcos(const TcArgs &a, const uint16_t *cv, int ldS, const double *cnorm, double *scores,
                          cudaStream_t st);
cudaError_t tc_cosine_read_status(cudaStream_t st, int *status);
// Status word of the auxiliary tensor-core kernels (packed Hamming, wait self-test).
cudaError_t tc_aux_read_status(cudaStream_t st, int *status);

}  // namespace hdc
