/*
 * hdc.h -- C ABI of libhdc, a GB300 (sm_103a) library for the data-parallel
 * hot path of hyperdimensional-computing (HDC) classification under the
 * approximation knobs studied in "Compiler-Driven Approximation Tuning for
 * Hyperdimensional Computing" (ApproxHDC).
 *
 * The path (Sec. 2.1; Listing 1):
 *   encode   h = sign(x . B)          random projection, __hetero_hdc_matmul
 *   pack     +-1 -> one bit per dim   Automatic Binarization (Sec. 4.2)
 *   compare  Hamming distance to C class hypervectors
 *            (or cosine on b-bit class hypervectors, "Algorithmic Choice")
 *   choose   arg-min / arg-max        __hetero_hdc_arg_min
 *   train    bundling + retraining    Sec. 2.1 training stage; TRAIN_ITERATIONS
 * and the knobs (Sec. 4.2): reduction perforation (start, end, stride) of the
 * dimension axis, element type of the encoding (FP32, BF16, FP8 E4M3) and of
 * the class hypervectors (1, 4 or 8 bits).
 *
 * CONVENTIONS (all entry points)
 *  - Every array argument is DEVICE memory owned by the caller unless the
 *    name says _host.  The library never allocates device memory, never
 *    frees, never synchronises the stream (except hdc_stream_status and the
 *    _host entry points, which say so) and keeps no state between calls.
 *  - Work is enqueued on `stream` (a cudaStream_t; NULL = legacy default).
 *    Results are valid once the stream has reached that point.
 *  - Row-major throughout.  A packed hypervector of L dimensions occupies
 *    W(L) = ceil(L/32) rounded up to a multiple of 4 uint32 words: bit d is
 *    bit (d % 32) of word d / 32, a set bit is the element -1, sign(0) = +1,
 *    and every bit past L is zero.  Packed rows are 16-byte aligned.
 *  - Arguments are checked before anything is enqueued: a NULL required
 *    pointer, a size out of range, a misaligned pointer or a workspace that
 *    is too small returns an error and enqueues nothing.  A failed launch
 *    returns HDC_ERR_CUDA.  Device-side failures (a bounded wait that ran out,
 *    a failed device check) set a device status word that hdc_stream_status
 *    reports; the library never traps, aborts or throws across this ABI.
 */
#ifndef HDC_H
#define HDC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *hdc_stream_t; /* same type as cudaStream_t */

typedef enum {
    HDC_OK = 0,
    HDC_ERR_INVALID_ARG = 1, /* NULL pointer, size out of range, misalignment */
    HDC_ERR_UNSUPPORTED = 2, /* valid but not built (e.g. class_bits = 3)     */
    HDC_ERR_WORKSPACE = 3,   /* caller buffer smaller than the size query     */
    HDC_ERR_CUDA = 4,        /* a CUDA runtime call or launch failed          */
    HDC_ERR_TIMEOUT = 5,     /* a bounded device wait expired                 */
    HDC_ERR_DEVICE = 6       /* a device-side check failed                    */
} hdc_status;

/* Element type of the encoding contraction (Sec. 4.2 "Element Type
 * Representation").  FP32: FFMA on CUDA cores, the plain exact form.
 * BF16: round-to-nearest-even, tensor cores, FP32 accumulation.
 * FP8_E4M3: per-row power-of-two scale s = smallest 2^k with amax <= 448*s
 * (rows of x and rows of B^T alike), round-to-nearest-even with saturation,
 * tensor cores, FP32 accumulation.  Positive scales leave sign(x.B) as is.  */
typedef enum {
    HDC_ENC_FP32 = 0,
    HDC_ENC_BF16 = 1,
    HDC_ENC_FP8_E4M3 = 2
} hdc_enc;

/* One approximation configuration (mirrors the per-operation JSON of
 * Listing 3: red_perf {base, stride, extent} plus an algorithmic choice).
 * Kept dimensions K = { s0 + k*stride : s0 + k*stride < e0 } with
 * s0 = floor(perf_start*D), e0 = floor(perf_end*D), both products in double
 * (Listing 1: red_perf(dists, 0.0, 0.5, 1) keeps the first half of D).
 * class_bits 1 = binary class hypervectors, Hamming distance, arg-min;
 * class_bits 4 or 8 = b-bit class hypervectors, cosine score, arg-max.     */
typedef struct {
    uint32_t struct_size; /* = sizeof(hdc_approx_config)                    */
    float perf_start;     /* in [0, 1)                                      */
    float perf_end;       /* in (perf_start, 1]                             */
    uint32_t perf_stride; /* >= 1                                           */
    int32_t enc;          /* hdc_enc                                        */
    uint32_t class_bits;  /* 1, 4 or 8                                      */
    uint32_t flags;       /* HDC_FLAG_* below                               */
    /* Reduction perforation of the encoding itself (the matmul over the F
     * features; Sec. 4.2, and what the paper's no-approx hint of Sec. 4.3
     * forbids): kept features s0 + k*stride < e0 with s0 = floor(start*F),
     * e0 = floor(end*F) as for the dims.  (0, 1, 1) keeps every feature.
     * Signs, class decisions and cosines do not depend on the rescaling
     * by F / F' that a perforated mat-vec estimate would take, so none is
     * applied; hdc_encode's optional projections are sums over the kept
     * features.                                                            */
    float enc_perf_start;
    float enc_perf_end;
    uint32_t enc_perf_stride;
} hdc_approx_config;

/* Force the CUDA-core (FFMA) encoder even for BF16/FP8 inputs.             */
#define HDC_FLAG_SIMT_ENCODE 0x1u

/* Float query hypervectors (Sec. 4.2 Algorithmic Choice: cosine similarity
 * on non-binarised hypervectors, the paper's float + cosine baselines of
 * Sec. 5.2).  The encoded query is not binarised: for each kept dim k,
 *   q_k = bf16( s_k * sb_k ),  s_k = sum_f x^_f b^_{k,f}
 * (sb_k the FP8 scale of base row k, 1 otherwise; the query row's scale is
 * a common positive factor and is dropped, since the cosine ignores it), and
 *   score_c = sum_k q_k c_k / ( ||q|| ||c|| )   (0 when a norm is 0)
 * against the b-bit class values c of class_bits 4 or 8 (the quantisation of
 * the binary path), FP32 tensor-core dot products, FP64 score, arg-max with
 * the lowest index on ties.  Requires class_bits 4 or 8 and C <= 256.       */
#define HDC_FLAG_FLOAT_QUERY 0x2u

/* Fill *cfg with the unapproximated configuration: perforation (0, 1, 1),
 * FP32 encoding, binary class hypervectors.                                */
void hdc_default_config(hdc_approx_config *cfg);

/* Number of kept dimensions |K| of cfg's perforation on D dims, or -1 if
 * the perforation arguments are invalid.  Host-only, no CUDA call.          */
int64_t hdc_kept_dims(int32_t D, const hdc_approx_config *cfg);

/* Words per packed row of L dimensions: ceil(L/32) rounded up to 4.         */
int32_t hdc_words(int32_t L);

/* A prepared model: views into a caller-owned device buffer filled by
 * hdc_model_prepare.  Read-only for every other entry point.               */
typedef struct {
    uint32_t struct_size;
    int32_t F;          /* features                                          */
    int32_t D;          /* full dimensionality                               */
    int32_t Dk;         /* kept dimensions |K|                               */
    int32_t C;          /* classes (0 = base only)                           */
    int32_t enc;        /* hdc_enc of Bq                                     */
    int32_t ldb;        /* elements per row of Bq (F rounded up, zero pad)   */
    int32_t class_bits; /* 1, 4 or 8                                         */
    int32_t W;          /* words per packed hypervector over Dk dims         */
    uint32_t flags;     /* HDC_FLAG_* of the configuration                   */
    const void *Bq;     /* Dk x ldb: rows K of B^T in the encoding type      */
    const float *b_scale;      /* Dk row scales (FP8) or NULL               */
    const uint32_t *cls;       /* class_bits planes, each C x W words;       */
                               /* plane j holds bit j of the two's-         */
                               /* complement class value (1 plane = sign)   */
    const int32_t *cls_sum;    /* C: sum over K of the class values (b > 1) */
    const double *cls_norm;    /* C: sqrt(sum over K of class value^2)       */
    const uint8_t *cls_sign;   /* binary classes, 33 <= C <= 112: Cp x ldcs  */
                               /* E4M3 +-1 bytes of the class hypervectors  */
                               /* (0 past Dk and for the pad classes up to  */
                               /* Cp = C rounded to 16) for the tensor-core */
                               /* Hamming distances; NULL otherwise         */
    int32_t ldcs;              /* bytes per row of cls_sign                 */
    int32_t Fk;                /* kept features F' (= F without encoding    */
                               /* perforation); Bq rows hold these          */
    int32_t fs0, fstride;      /* kept feature k is column fs0 + k*fstride  */
} hdc_model;

/* Bytes of device buffer hdc_model_prepare needs for this configuration.  */
hdc_status hdc_model_bytes(int32_t F, int32_t D, int32_t C,
                           const hdc_approx_config *cfg, size_t *bytes);

/* Prepare a model for cfg (model load, Sec. 4.2 knobs applied once):
 *  - rows K of Bt (D x F FP32, the transposed base hypermatrix, Listing 1
 *    rp_matrix) are gathered, quantised to cfg->enc and zero-padded to ldb;
 *  - if acc (C x D int32 class accumulators from hdc_train_epoch) is not
 *    NULL, the class hypervectors are quantised to cfg->class_bits over ALL
 *    D dims (b = 1: sign; b > 1: per class Q = 2^(b-1)-1, M = max|acc|,
 *    value = sign(acc)*floor((2|acc|Q + M)/(2M)), 0 if M = 0), restricted
 *    to K, and stored as bit planes with their sums and norms over K.
 * buf (>= hdc_model_bytes, 256-byte aligned) receives all data; *out gets
 * the views.  C may be 0 (with acc NULL) for a base-only model.          */
hdc_status hdc_model_prepare(const float *Bt, int32_t F, int32_t D,
                             const int32_t *acc, int32_t C,
                             const hdc_approx_config *cfg, void *buf,
                             size_t buf_bytes, hdc_model *out,
                             hdc_stream_t stream);

/* Workspace bytes for hdc_encode / hdc_classify on N query rows.         */
hdc_status hdc_workspace_bytes(int64_t N, const hdc_model *m, size_t *bytes);

/* Encode (Listing 1 __hetero_hdc_matmul + Automatic Binarization):
 * H[i] = pack(sign(X[i] . B[:, K]))  for X (N x F FP32, rows 16-byte
 * aligned when F % 4 == 0).  H is N x m->W words.  If scores is not NULL
 * it receives the N x Dk FP32 projections (de-scaled: x . B estimate), for
 * parity checks.  ws: >= hdc_workspace_bytes(N, m), 256-byte aligned.   */
hdc_status hdc_encode(const float *X, int64_t N, const hdc_model *m,
                      uint32_t *H, float *scores, void *ws, size_t ws_bytes,
                      hdc_stream_t stream);

/* Hamming distance + arg-min (Listing 1: __hetero_hdc_hamming_distance,
 * red_perf, __hetero_hdc_arg_min) on packed hypervectors of D dims:
 * dist[i][c] = number of kept dims d in K(cfg, D) with Q[i] and Cls[c]
 * different; labels[i] = arg-min, lowest class index on ties.  Q is N x
 * W(D), Cls is C x W(D).  dists (N x C int32) is optional.  Only the
 * perforation fields of cfg are used (NULL = no perforation).            */
hdc_status hdc_hamming_argmin(const uint32_t *Q, const uint32_t *Cls,
                              int64_t N, int32_t C, int32_t D,
                              const hdc_approx_config *cfg, int32_t *labels,
                              int32_t *dists, hdc_stream_t stream);

/* Workspace bytes for hdc_hamming_argmin_ws: for 33..256 classes and
 * D <= 131072 (the tensor-core route), the class hypervectors expanded to
 * one E4M3 +-1 byte per dim (C rounded up to 16 rows of
 * 256 * ceil(W(D) / 8) bytes); 0 for every other C and D.
 * HDC_ERR_INVALID_ARG for C <= 0, D <= 0 or a NULL bytes.                  */
hdc_status hdc_hamming_argmin_workspace_bytes(int32_t C, int32_t D, size_t *bytes);

/* hdc_hamming_argmin (same definition, arguments and results) with a
 * caller workspace ws of ws_bytes (device, 256-byte aligned, caller-owned,
 * >= hdc_hamming_argmin_workspace_bytes(C, D); NULL when that is 0).  On
 * the tensor-core route the class hypervectors are expanded into ws once
 * per call instead of once per 128-row tile.  HDC_ERR_WORKSPACE when ws is
 * too small or misaligned; it is overwritten (no result lives in it).     */
hdc_status hdc_hamming_argmin_ws(const uint32_t *Q, const uint32_t *Cls,
                                 int64_t N, int32_t C, int32_t D,
                                 const hdc_approx_config *cfg, int32_t *labels,
                                 int32_t *dists, void *ws, size_t ws_bytes,
                                 hdc_stream_t stream);

/* Workspace bytes for hdc_train_epoch (about 12 N + 32 C bytes): the N
 * predictions of a retraining epoch, a 2N-entry permutation grouping the
 * samples (a misclassified sample sits in its true class's group and in its
 * predicted class's), and per-group (2C) counts, offsets, first counting
 * items and cursors.  HDC_ERR_INVALID_ARG for N < 0, D <= 0, C <= 0 or a
 * NULL bytes; HDC_ERR_UNSUPPORTED for N > 2^30 - 1 or C > 2^28 (the
 * grouping's int32 offsets cover 2N entries).                              */
hdc_status hdc_train_workspace_bytes(int64_t N, int32_t D, int32_t C,
                                     size_t *bytes);

/* One training pass over N packed training hypervectors H (N x W(D)) with
 * labels y (int32 in [0, C); other labels are skipped):
 *  mode 0 (bundling, Sec. 2.1): acc[c][d] = sum over n with y_n = c of
 *         (1 - 2*bit[n][d])   (acc is overwritten);
 *  mode 1 (retraining epoch, TRAIN_ITERATIONS): every sample is classified
 *         by Hamming arg-min against cls as it is on entry; then, for each
 *         misclassified n, acc[y_n] += h_n and acc[pred_n] -= h_n with
 *         h = 1 - 2*bit (perceptron, applied once per epoch);
 *  mode 2 (the retraining delta of one shard of the samples): as mode 1,
 *         but acc is overwritten with the updates alone (acc = 0 plus the
 *         +h_n / -h_n of this call's misclassified samples) and cls is left
 *         as it is.  Shards that share the start-of-epoch cls and sum their
 *         deltas (an integer all-reduce) reproduce mode 1 over all samples
 *         exactly; hdc_train_apply then adds the sum and re-binarises.
 * In modes 0 and 1 cls (C x W(D)) is then rewritten as the sign of acc.
 * n_updates (one int32, device, optional) receives the number of updates.
 * acc (C x D int32) must not overflow: |acc| < 2^31.  All pointers are
 * caller-owned device memory: H and cls 16-byte aligned, ws (>=
 * hdc_train_workspace_bytes(N, D, C), 256-byte aligned) scratch for this
 * call only.  Errors: HDC_ERR_INVALID_ARG (sizes, mode, NULL or misaligned
 * pointers), HDC_ERR_UNSUPPORTED (N > 2^30 - 1 or C > 2^28),
 * HDC_ERR_WORKSPACE (ws too small or misaligned), HDC_ERR_CUDA; nothing is
 * enqueued on an argument error.                                          */
hdc_status hdc_train_epoch(const uint32_t *H, const int32_t *y, int64_t N,
                           int32_t D, int32_t C, int32_t mode, int32_t *acc,
                           uint32_t *cls, int32_t *n_updates, void *ws,
                           size_t ws_bytes, hdc_stream_t stream);

/* The exchange step of training over sharded samples (Sec. 2.1 training;
 * TRAIN_ITERATIONS epochs, each epoch's updates applied at once):
 * acc[c][d] += delta[c][d] (skipped when delta is NULL), then cls (C x W(D))
 * = pack(acc < 0), the sign of the bundle.  After per-shard bundles (mode 0)
 * are summed into acc, delta = NULL binarises the sum; after per-shard
 * deltas (mode 2) are summed into delta, this applies the epoch.  acc and
 * delta are C x D int32 device arrays (|acc + delta| < 2^31), cls is device
 * memory, 16-byte aligned.  Errors: HDC_ERR_INVALID_ARG (C <= 0, D <= 0,
 * NULL acc or cls, misaligned cls), HDC_ERR_CUDA; nothing is enqueued on an
 * argument error.                                                         */
hdc_status hdc_train_apply(const int32_t *delta, int32_t C, int32_t D,
                           int32_t *acc, uint32_t *cls, hdc_stream_t stream);

/* Classify (Listing 1 end to end under the model's knobs):
 * labels[i] for X (N x F FP32).  class_bits 1: Hamming arg-min over K,
 * dists (N x C int32, optional).  class_bits > 1: cosine arg-max with
 * score = dot(1-2*q, chat) / ||chat|| over K (IEEE FP64, 0 if the norm is
 * 0), scores (N x C double, optional).  Encoded hypervectors are kept on
 * chip on the tensor-core path and never written to memory.              */
hdc_status hdc_classify(const float *X, int64_t N, const hdc_model *m,
                        int32_t *labels, int32_t *dists, double *scores,
                        void *ws, size_t ws_bytes, hdc_stream_t stream);

/* hdc_classify for query rows in HOST memory: the n_parts row blocks
 * parts_host[i] (part_rows[i] x m->F FP32 each, contiguous; page-locked for
 * the copies to overlap other work) are copied in order into X_dev (device,
 * sum(part_rows) x F FP32), classified with workspace ws as hdc_classify
 * does, and the labels (device labels_dev, sum(part_rows) int32) are copied
 * back to labels_host.  Everything is enqueued on `stream`; host buffers
 * must stay valid and unmodified until the stream reaches this point.
 * Used by the serving loop (one call per batch) and for end-to-end timing. */
hdc_status hdc_classify_host(const float *const *parts_host, const int64_t *part_rows,
                             int32_t n_parts, const hdc_model *m, float *X_dev,
                             int32_t *labels_dev, int32_t *labels_host, void *ws,
                             size_t ws_bytes, hdc_stream_t stream);

/* Batched evaluation of approximation configurations.  The paper's tuner
 * (Sec. 3, Fig. 1) compiles and runs the application once per candidate
 * configuration and reads back its QoS (accuracy).  Here every combination
 * of perforation entry x class-hypervector width of one trained model is
 * scored in one launch from the same validation hypervectors encoded once
 * at the full D: every entry's kept dimensions are one 32-bit mask pattern
 * per word (stride a power of two <= 32), cut at the entry's first and last
 * word, so all configurations share the same loads.
 *   entry i     the perforation (starts[i], ends[i], strides[i]) of
 *               hdc_classify: with s0 = floor(starts[i]*D) and
 *               e0 = floor(ends[i]*D) (both formed in double), the kept
 *               dims are d = s0 + k*strides[i] < e0
 *   strides[i]  power of two <= 32
 *   starts[i]   start fraction in [0, 1)
 *   ends[i]     end fraction in (0, 1] (0 means 1.0); e0 > s0 is required
 *   bits[j]     1 (Hamming, arg-min), 4 or 8 (b-bit cosine, arg-max, as in
 *               hdc_classify), or 0: cosine against the unquantised int32
 *               accumulators themselves (requires sum over D of acc^2 < 2^63)
 * block_threads / words_per_chunk are launch-shape knobs (0 = default;
 * 64, 128 or 256 threads; a multiple of 4 words) chosen by an autotuner;
 * results do not depend on them.                                           */
#define HDC_SWEEP_MAX_STRIDES 6
#define HDC_SWEEP_MAX_BITS 4
typedef struct {
    uint32_t struct_size;                 /* = sizeof(hdc_sweep_spec)       */
    int32_t n_strides;                    /* 1 .. HDC_SWEEP_MAX_STRIDES     */
    int32_t strides[HDC_SWEEP_MAX_STRIDES];
    float starts[HDC_SWEEP_MAX_STRIDES];
    float ends[HDC_SWEEP_MAX_STRIDES];
    int32_t n_bits;                       /* 1 .. HDC_SWEEP_MAX_BITS        */
    int32_t bits[HDC_SWEEP_MAX_BITS];
    int32_t block_threads;                /* 0, 64, 128 or 256              */
    int32_t words_per_chunk;              /* 0 or a multiple of 4           */
} hdc_sweep_spec;

/* Workspace bytes for hdc_sweep_eval.                                      */
hdc_status hdc_sweep_workspace_bytes(int32_t D, int32_t C, const hdc_sweep_spec *spec,
                                     size_t *bytes);

/* Score every (bits[j], strides[i]) configuration: H (N x W(D) packed
 * validation hypervectors encoded at the full D, any encoding type), y (N
 * labels), acc (C x D class accumulators).  correct (n_bits x n_strides
 * int32, overwritten) counts the queries whose predicted class equals y;
 * labels (optional, n_bits x n_strides x N int32) receives the predictions,
 * which equal hdc_classify's for the same model and configuration.        */
hdc_status hdc_sweep_eval(const uint32_t *H, const int32_t *y, int64_t N, int32_t D,
                          int32_t C, const int32_t *acc, const hdc_sweep_spec *spec,
                          int32_t *correct, int32_t *labels, void *ws, size_t ws_bytes,
                          hdc_stream_t stream);

/* Level-ID encoding (Sec. 4.2 Algorithmic Choice: ID-based encoding as the
 * alternative to random projection; Sec. 5.3: Micro-HD-Classification's
 * encoder, with its N_LEVELS knob L).  Packed bits use the convention of the
 * rest of the ABI: bit 1 = element -1.
 *   level(x_f) = clamp(floor((x_f - lo) * scale), 0, L-1), the difference
 *                and the product each rounded to FP32 (no fused multiply-
 *                add), NaN -> level 0; scale = (float)(L / (x_hi - x_lo))
 *                formed in double
 *   LEVEL_l[d] = hi_hv[d] if l >= flip[d] else lo_hv[d]   (flip[d] in
 *                1..L-1: level 0 is lo_hv, level L-1 is hi_hv)
 *   s_d        = sum_f ID_f[d] * LEVEL_{level(x_f)}[d],  bit_d = s_d < 0
 * over the kept dims of cfg's perforation (compacted at preparation, as
 * for the random projection; enc, class_bits and flags are not used).
 * The encoded rows feed hdc_train_epoch / hdc_hamming_argmin / hdc_cluster
 * with D = Dk.  Limits: F < 8192 and (F + L) * 128 bytes <= 200 KB.       */
typedef struct {
    uint32_t struct_size;        /* = sizeof(hdc_levelid_model)             */
    int32_t F, D, Dk, L, W;      /* W = hdc_words(Dk)                       */
    float lo, scale;
    const uint32_t *id;          /* F x W packed ID hypervectors (kept dims) */
    const uint32_t *level;       /* L x W packed level hypervectors         */
} hdc_levelid_model;

/* Bytes of the model buffer (256-byte aligned, caller-owned).             */
hdc_status hdc_levelid_model_bytes(int32_t F, int32_t D, int32_t L, const hdc_approx_config *cfg,
                                   size_t *bytes);

/* Build a Level-ID model in buf: the kept dims of the ID and level
 * hypervectors, packed.  Device inputs, one byte per element (nonzero = the
 * element -1, zero = +1): id_bits (F x D, row-major), lo_bits and hi_bits
 * (D each, the two level end points); flip (D int32).  The random
 * hypervectors and flip levels are the caller's draws.  flip_error
 * (optional device int32) is set to 1 if some flip[d] is outside 1..L-1.
 * Errors: HDC_ERR_INVALID_ARG (sizes, pointers, x_hi <= x_lo, non-finite
 * bounds), HDC_ERR_UNSUPPORTED (limits), HDC_ERR_WORKSPACE, HDC_ERR_CUDA. */
hdc_status hdc_levelid_prepare(const uint8_t *id_bits, const uint8_t *lo_bits, const uint8_t *hi_bits,
                               const int32_t *flip, int32_t F, int32_t D, int32_t L, float x_lo,
                               float x_hi, const hdc_approx_config *cfg, void *buf, size_t buf_bytes,
                               int32_t *flip_error, hdc_levelid_model *out, hdc_stream_t stream);

/* Encode N rows of X (N x F FP32, device) into H (N x W packed, device).   */
hdc_status hdc_levelid_encode(const float *X, int64_t N, const hdc_levelid_model *m, uint32_t *H,
                              hdc_stream_t stream);

/* HD-Clustering (Sec. 5.1): K-means over binary hypervectors.  The paper's
 * benchmark clusters encoded points with K cluster hypervectors, refining
 * them for TRAIN_ITERATIONS iterations, and scores the result by NMI; its
 * two similarity ops (training and inference) are tuned independently.
 * One iteration:
 *   assign  label[n] = arg-min_k Hamming(H[n], cls[k]) over the kept dims of
 *           train_sim's perforation (lowest k on ties);
 *   update  acc[k] = sum over the members n of (1 - 2*bit_n) over all D,
 *           cls[k] = (acc[k] < 0) -- a cluster without members becomes all
 *           +1 (bit 0), as sign(0) = +1.
 * After `iters` iterations, labels = the assignment under infer_sim.
 *   H        N x W(D) packed point hypervectors (device, 16-byte aligned)
 *   cls      K x W(D) packed cluster hypervectors: the initial ones on
 *            entry (e.g. K distinct points), the final ones on return
 *   acc      K x D int32 (out): the accumulators of the last update
 *            (untouched when iters = 0)
 *   labels   N int32 (out)
 *   changes  optional int32[iters] (out): points whose cluster differs
 *            from the previous iteration's (iteration 0: N)
 *   train_sim, infer_sim  perforation (perf_start, perf_end, perf_stride)
 *            of the two similarity ops; NULL = all D; class_bits must be 1
 *            (enc is not used)
 *   ws       hdc_cluster_workspace_bytes(N, D, K) bytes, 256-byte aligned
 * Errors: HDC_ERR_INVALID_ARG (sizes, pointers, a perforation that keeps
 * nothing), HDC_ERR_UNSUPPORTED (N > 2^30 - 1 or K > 2^28, as training),
 * HDC_ERR_WORKSPACE, HDC_ERR_CUDA.                                         */
hdc_status hdc_cluster_workspace_bytes(int64_t N, int32_t D, int32_t K, size_t *bytes);
hdc_status hdc_cluster(const uint32_t *H, int64_t N, int32_t D, int32_t K, int32_t iters,
                       const hdc_approx_config *train_sim, const hdc_approx_config *infer_sim,
                       uint32_t *cls, int32_t *acc, int32_t *labels, int32_t *changes, void *ws,
                       size_t ws_bytes, hdc_stream_t stream);

/* Size of the fixed scratch array behind hdc_classify_static.              */
#define HDC_STATIC_SCRATCH_BYTES ((size_t)64 << 20)

/* hdc_classify for callers that cannot allocate device memory.  The paper
 * has no counterpart; this is a deployment convenience.  A plugin inside a
 * serving process whose device memory belongs to another allocator, a
 * process held to a device-memory budget fixed at start-up, or a loop that
 * may not call cudaMalloc (it can synchronise the device) passes only its
 * inputs and outputs; the scratch that hdc_classify takes as `ws` is a
 * fixed device array compiled into the library instead.
 *  - Limit: calls with hdc_workspace_bytes(N, m) > HDC_STATIC_SCRATCH_BYTES
 *    (64 MiB: about 31,000 queries of 784 features at 10,000 dims) return
 *    HDC_ERR_WORKSPACE and enqueue nothing; split larger batches.
 *  - Every GPU that loads libhdc holds the array until the process exits.
 *  - The first call on a device looks up the array's device address (set-up,
 *    once per device, with that device current); make that first call
 *    before any stream capture.
 *  - Every call shares the one array, which keeps the last call's contents
 *    (nothing in it needs to start at zero).  Calls whose work overlaps on
 *    the GPU -- e.g. on two streams without ordering -- race on it: order
 *    them on one stream or with events.
 * Arguments, outputs and errors are otherwise those of hdc_classify; the
 * library allocates nothing.                                              */
hdc_status hdc_classify_static(const float *X, int64_t N, const hdc_model *m,
                               int32_t *labels, int32_t *dists, double *scores,
                               hdc_stream_t stream);

/* Waits for `stream`, then reads and clears the library's device status
 * words: HDC_OK, HDC_ERR_TIMEOUT or HDC_ERR_DEVICE (or HDC_ERR_CUDA if the
 * stream itself reports an error).                                        */
hdc_status hdc_stream_status(hdc_stream_t stream);

/* Failure-detection self-test (not part of the method).  Enqueues one
 * 32-thread block that waits on a shared-memory barrier nothing arrives
 * on, through the same bounded-wait routine the tensor-core kernels use,
 * with a limit of `limit_us` microseconds (1 .. 2,000,000).  The wait runs
 * out, the block records a timeout in the device status word and returns:
 * the next hdc_stream_status on `stream` returns HDC_ERR_TIMEOUT, and the
 * context stays usable.  Nothing faults, traps or hangs.  Returns
 * HDC_ERR_INVALID_ARG for a limit out of range (nothing enqueued),
 * HDC_ERR_CUDA if the launch fails, else HDC_OK.                          */
hdc_status hdc_selftest_wait(uint32_t limit_us, hdc_stream_t stream);

/* Tracing hook (not part of the method): with start and stop set to
 * cudaEvent_t handles, every later hdc_encode / hdc_classify call made by
 * the calling host thread records `start` on its stream just before its
 * encoding kernel and `stop` just after it, so that kernel can be timed on
 * its own with cudaEventElapsedTime.  The handles stay owned by the caller;
 * hdc_profile_events(NULL, NULL) turns the hook off.                        */
void hdc_profile_events(void *start, void *stop);

/* Static English text for a status code.                                   */
const char *hdc_status_string(hdc_status s);

#ifdef __cplusplus
}
#endif
#endif /* HDC_H */
