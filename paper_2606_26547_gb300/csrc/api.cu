// C-ABI entry points of libhdc (declared and documented in include/hdc.h):
// argument checks, carving of caller-owned buffers, and the launch sequence
// of each call.  Every step of the path runs in the library's kernels.
#include <math.h>
#include <string.h>

#include "hdc_internal.cuh"

namespace hdc {

bool perf_of(int64_t D, const hdc_approx_config *cfg, Perf *p)
{
    float st = 0.f, en = 1.f;
    int64_t stride = 1;
    if (cfg) {
        st = cfg->perf_start;
        en = cfg->perf_end;
        stride = cfg->perf_stride;
    }
    if (D <= 0 || stride < 1 || !(st >= 0.f) || !(en <= 1.f) || !(st < en)) return false;
    p->s0 = (int64_t)floor((double)st * (double)D);
    p->e0 = (int64_t)floor((double)en * (double)D);
    p->stride = stride;
    p->Dk = p->e0 > p->s0 ? (p->e0 - p->s0 + stride - 1) / stride : 0;
    return p->Dk > 0;
}

// Kept features of the encoding's perforation (the same rule over F).
bool feat_perf_of(int64_t F, const hdc_approx_config *cfg, Perf *p)
{
    hdc_approx_config c;
    hdc_default_config(&c);
    if (cfg) {
        c.perf_start = cfg->enc_perf_start;
        c.perf_end = cfg->enc_perf_end;
        c.perf_stride = cfg->enc_perf_stride;
    }
    return perf_of(F, &c, p);
}

namespace {

inline bool aligned(const void *p, size_t a) { return ((uintptr_t)p % a) == 0; }

bool cfg_ok(const hdc_approx_config *cfg)
{
    if (!cfg || cfg->struct_size < sizeof(hdc_approx_config)) return false;
    if (cfg->enc < HDC_ENC_FP32 || cfg->enc > HDC_ENC_FP8_E4M3) return false;
    return true;
}

bool bits_ok(uint32_t b) { return b == 1 || b == 4 || b == 8; }

bool float_query(uint32_t flags) { return (flags & HDC_FLAG_FLOAT_QUERY) != 0; }

// The float-query path: cosine on b-bit classes, at most 256 of them.
bool flags_ok(uint32_t flags, uint32_t bits, int C)
{
    if (flags & ~(HDC_FLAG_SIMT_ENCODE | HDC_FLAG_FLOAT_QUERY)) return false;
    return !float_query(flags) || (bits > 1 && C <= 256);
}

// Row length (BF16 elements) of the float projections and class values.
inline int lds_for(int Dk) { return ld_for(HDC_ENC_BF16, Dk); }
inline int cpad_for(int C) { return (C + 15) / 16 * 16; }

bool model_ok(const hdc_model *m)
{
    return m && m->struct_size >= sizeof(hdc_model) && m->F > 0 && m->D > 0 && m->Dk > 0 && m->Dk <= m->D &&
           m->Fk > 0 && m->Fk <= m->F && m->fs0 >= 0 && m->fstride >= 1 &&
           m->fs0 + (int64_t)(m->Fk - 1) * m->fstride < m->F &&
           m->C >= 0 && m->Bq && m->ldb >= m->Fk && m->W == words_for(m->Dk) && bits_ok((uint32_t)m->class_bits) &&
           m->enc >= HDC_ENC_FP32 && m->enc <= HDC_ENC_FP8_E4M3 && (m->enc != HDC_ENC_FP8_E4M3 || m->b_scale) &&
           flags_ok(m->flags, (uint32_t)m->class_bits, m->C);
}

struct ModelLayout {
    size_t bq, bscale, planes, csum, cnorm, csign, total;
};

// Binary classes with 33 <= C <= 112 also keep E4M3 +-1 class bytes for the
// tensor-core Hamming distances: Cp rows (C rounded to 16) of one byte per
// kept dim, padded to whole 192-dim tiles plus the 64 bytes the last tile's
// second 128-byte box reaches past them.
inline bool tc_hamming_classes(int bits, int C, uint32_t flags)
{
    return bits == 1 && C > 32 && C <= 112 && !(flags & HDC_FLAG_FLOAT_QUERY);
}
inline int ldcs_for(int Dk) { return (Dk + 191) / 192 * 192 + 64; }

ModelLayout model_layout(int F, int Dk, int C, int enc, int bits, uint32_t flags)
{
    ModelLayout L;
    size_t off = 0;
    const int ldb = ld_for(enc, F), W = words_for(Dk);
    // binary queries: b planes [b][C][W]; float queries: Cp x ldS BF16 values
    const size_t cls_bytes = float_query(flags) ? (size_t)cpad_for(C) * lds_for(Dk) * 2 : (size_t)bits * C * W * 4;
    L.bq = off;     off = align_up(off + (size_t)Dk * ldb * esize_for(enc), kAlign);
    L.bscale = off; off = align_up(off + (enc == HDC_ENC_FP8_E4M3 ? (size_t)Dk * 4 : 0), kAlign);
    L.planes = off; off = align_up(off + cls_bytes, kAlign);
    L.csum = off;   off = align_up(off + (size_t)C * 4, kAlign);
    L.cnorm = off;  off = align_up(off + (size_t)C * 8, kAlign);
    L.csign = off;
    off = align_up(off + (tc_hamming_classes(bits, C, flags) ? (size_t)cpad_for(C) * ldcs_for(Dk) : 0), kAlign);
    L.total = off;
    return L;
}

struct WsLayout {
    size_t xq, sx, h, sp, qn, sf, dacc, csign, total;
};

// Binary classes past the fused kernels (129..256): the classify's Hamming
// step expands the class hypervectors once per call into the workspace for
// the tensor-core route (0 bytes where that route does not apply).
size_t classify_sign_bytes(const hdc_model *m)
{
    if (m->class_bits != 1 || m->C <= 128 || float_query(m->flags)) return 0;
    return class_sign_bytes(m->C, m->W);
}

bool use_tc(const hdc_model *m);

WsLayout ws_layout(int64_t N, const hdc_model *m)
{
    WsLayout L;
    size_t off = 0;
    const bool quant = m->enc != HDC_ENC_FP32;
    const bool gather = m->Fk != m->F;   // perforated encoding: the kept features are gathered first
    const int ldx = ld_for(m->enc, m->Fk);
    const bool fq = float_query(m->flags);
    L.xq = off; off = align_up(off + (quant || gather ? (size_t)N * ldx * esize_for(m->enc) : 0), kAlign);
    L.sx = off; off = align_up(off + (m->enc == HDC_ENC_FP8_E4M3 ? (size_t)N * 4 : 0), kAlign);
    L.h = off;  off = align_up(off + (size_t)N * m->W * 4, kAlign);
    // float queries: BF16 projections and their norms; FP32 projections
    // first when the CUDA-core encoder computes them
    L.sp = off; off = align_up(off + (fq ? (size_t)N * lds_for(m->Dk) * 2 : 0), kAlign);
    L.qn = off; off = align_up(off + (fq ? (size_t)N * 4 : 0), kAlign);
    L.sf = off; off = align_up(off + (fq ? (size_t)N * m->Dk * 4 : 0), kAlign);
    // a classify of few query tiles splits their dim tiles over CTAs: the
    // partial distances of at most TC_SPLIT_MAX_TILES tiles and their counters
    L.dacc = off;
    off = align_up(off + (m->C > 0 && !fq ? tc_split_bytes(N, m->C) : 0), kAlign);
    L.csign = off; off = align_up(off + classify_sign_bytes(m), kAlign);
    L.total = off;
    return L;
}

hdc_status cu(cudaError_t e) { return e == cudaSuccess ? HDC_OK : HDC_ERR_CUDA; }

// Quantise X into the workspace (BF16/FP8); returns the operand to encode.
hdc_status prepare_queries(const float *X, int64_t N, const hdc_model *m, char *ws, const WsLayout &L,
                           const void **Xop, int64_t *ldx, const float **sx, cudaStream_t st)
{
    if (m->enc == HDC_ENC_FP32 && m->Fk == m->F) {
        *Xop = X;
        *ldx = m->F;
        *sx = nullptr;
        return HDC_OK;
    }
    // quantise (and, for a perforated encoding, gather the kept features)
    const int ld = ld_for(m->enc, m->Fk);
    float *scale = m->enc == HDC_ENC_FP8_E4M3 ? (float *)(ws + L.sx) : nullptr;
    hdc_status s = cu(launch_quant_rows(X, m->F, 0, 1, N, m->Fk, m->enc, ws + L.xq, ld, scale, st, m->fs0,
                                        m->fstride));
    *Xop = ws + L.xq;
    *ldx = ld;
    *sx = scale;
    return s;
}

// Tensor-core encoder for BF16/FP8 unless the configuration forces FFMA.
bool use_tc(const hdc_model *m) { return m->enc != HDC_ENC_FP32 && !(m->flags & HDC_FLAG_SIMT_ENCODE); }

// Tracing hook (hdc_profile_events): events recorded around the encoding
// kernel of each call made by this host thread.
thread_local cudaEvent_t t_prof_start = nullptr, t_prof_stop = nullptr;

cudaError_t timed_tc(const TcArgs &a, cudaStream_t st)
{
    if (t_prof_start) cudaEventRecord(t_prof_start, st);
    cudaError_t e = launch_tc_encode(a, st);
    if (t_prof_stop) cudaEventRecord(t_prof_stop, st);
    return e;
}

cudaError_t timed_simt(const void *X, int64_t ldx, int64_t N, int F, const void *Bq, int ldb, int Dk, int enc,
                       const float *sx, const float *sb, uint32_t *H, int W, float *scores, cudaStream_t st)
{
    if (t_prof_start) cudaEventRecord(t_prof_start, st);
    cudaError_t e = launch_encode_simt(X, ldx, N, F, Bq, ldb, Dk, enc, sx, sb, H, W, scores, st);
    if (t_prof_stop) cudaEventRecord(t_prof_stop, st);
    return e;
}

}  // namespace
}  // namespace hdc

using namespace hdc;

extern "C" {

void hdc_default_config(hdc_approx_config *cfg)
{
    if (!cfg) return;
    memset(cfg, 0, sizeof(*cfg));
    cfg->struct_size = sizeof(*cfg);
    cfg->perf_start = 0.f;
    cfg->perf_end = 1.f;
    cfg->perf_stride = 1;
    cfg->enc = HDC_ENC_FP32;
    cfg->class_bits = 1;
    cfg->flags = 0;
    cfg->enc_perf_start = 0.f;
    cfg->enc_perf_end = 1.f;
    cfg->enc_perf_stride = 1;
}

int64_t hdc_kept_dims(int32_t D, const hdc_approx_config *cfg)
{
    Perf p;
    if (cfg && cfg->struct_size < sizeof(hdc_approx_config)) return -1;
    return perf_of(D, cfg, &p) ? p.Dk : -1;
}

int32_t hdc_words(int32_t L) { return L < 0 ? -1 : words_for(L); }

hdc_status hdc_model_bytes(int32_t F, int32_t D, int32_t C, const hdc_approx_config *cfg, size_t *bytes)
{
    Perf p;
    if (!bytes || F <= 0 || D <= 0 || C < 0 || !cfg_ok(cfg) || !perf_of(D, cfg, &p)) return HDC_ERR_INVALID_ARG;
    if (!bits_ok(cfg->class_bits) || !flags_ok(cfg->flags, cfg->class_bits, C)) return HDC_ERR_UNSUPPORTED;
    Perf pf;
    if (!feat_perf_of(F, cfg, &pf)) return HDC_ERR_INVALID_ARG;
    *bytes = model_layout((int)pf.Dk, (int)p.Dk, C, cfg->enc, (int)cfg->class_bits, cfg->flags).total;
    return HDC_OK;
}

hdc_status hdc_model_prepare(const float *Bt, int32_t F, int32_t D, const int32_t *acc, int32_t C,
                             const hdc_approx_config *cfg, void *buf, size_t buf_bytes, hdc_model *out,
                             hdc_stream_t stream)
{
    Perf p;
    if (!Bt || !buf || !out || F <= 0 || D <= 0 || C < 0 || (C > 0 && !acc) || !cfg_ok(cfg) ||
        !perf_of(D, cfg, &p) || !aligned(buf, kAlign))
        return HDC_ERR_INVALID_ARG;
    if (!bits_ok(cfg->class_bits) || !flags_ok(cfg->flags, cfg->class_bits, C)) return HDC_ERR_UNSUPPORTED;
    Perf pf;
    if (!feat_perf_of(F, cfg, &pf)) return HDC_ERR_INVALID_ARG;
    const int Dk = (int)p.Dk, enc = cfg->enc, bits = (int)cfg->class_bits, Fk = (int)pf.Dk;
    const ModelLayout L = model_layout(Fk, Dk, C, enc, bits, cfg->flags);
    if (buf_bytes < L.total) return HDC_ERR_WORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    char *b = (char *)buf;
    hdc_model m;
    memset(&m, 0, sizeof(m));
    m.struct_size = sizeof(hdc_model);
    m.F = F;
    m.D = D;
    m.Dk = Dk;
    m.C = C;
    m.enc = enc;
    m.ldb = ld_for(enc, Fk);
    m.Fk = Fk;
    m.fs0 = (int32_t)pf.s0;
    m.fstride = (int32_t)pf.stride;
    m.class_bits = bits;
    m.flags = cfg->flags;
    m.W = words_for(Dk);
    m.Bq = b + L.bq;
    m.b_scale = enc == HDC_ENC_FP8_E4M3 ? (const float *)(b + L.bscale) : nullptr;
    // rows K of B^T: row k of Bq = quantise(Bt[s0 + k*stride])
    // rows K of B^T (and, for a perforated encoding, their kept features)
    hdc_status s = cu(launch_quant_rows(Bt, F, p.s0, p.stride, Dk, Fk, enc, b + L.bq, m.ldb,
                                        (float *)(b + L.bscale), st, pf.s0, pf.stride));
    if (s != HDC_OK) return s;
    if (C > 0) {
        m.cls = (const uint32_t *)(b + L.planes);
        m.cls_sum = (const int32_t *)(b + L.csum);
        m.cls_norm = (const double *)(b + L.cnorm);
        if (float_query(cfg->flags)) {
            // rows past C stay zero (the cosine kernel reads Cp rows)
            s = cu(cudaMemsetAsync(b + L.planes, 0, L.csum - L.planes, st));
            if (s != HDC_OK) return s;
        }
        s = cu(launch_class_prepare(acc, C, D, p, bits, (uint32_t *)(b + L.planes), m.W, (int32_t *)(b + L.csum),
                                    (double *)(b + L.cnorm),
                                    float_query(cfg->flags) ? (uint16_t *)(b + L.planes) : nullptr, lds_for(Dk),
                                    st));
        if (s != HDC_OK) return s;
        if (tc_hamming_classes(bits, C, cfg->flags)) {
            m.cls_sign = (const uint8_t *)(b + L.csign);
            m.ldcs = ldcs_for(Dk);
            s = cu(launch_class_sign((const uint32_t *)(b + L.planes), C, m.W, Dk, cpad_for(C), m.ldcs,
                                     (uint8_t *)(b + L.csign), st));
            if (s != HDC_OK) return s;
        }
    }
    *out = m;
    return HDC_OK;
}

hdc_status hdc_workspace_bytes(int64_t N, const hdc_model *m, size_t *bytes)
{
    if (!bytes || N < 0 || !model_ok(m)) return HDC_ERR_INVALID_ARG;
    *bytes = ws_layout(N, m).total;
    return HDC_OK;
}

hdc_status hdc_encode(const float *X, int64_t N, const hdc_model *m, uint32_t *H, float *scores, void *ws,
                      size_t ws_bytes, hdc_stream_t stream)
{
    if (N < 0 || !model_ok(m)) return HDC_ERR_INVALID_ARG;
    if (N == 0) return HDC_OK;
    if (!X || !H || !aligned(H, 16) || (ws_bytes && !ws) || (ws && !aligned(ws, kAlign))) return HDC_ERR_INVALID_ARG;
    const WsLayout L = ws_layout(N, m);
    if (ws_bytes < L.total) return HDC_ERR_WORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    const void *Xop;
    int64_t ldx;
    const float *sx;
    hdc_status s = prepare_queries(X, N, m, (char *)ws, L, &Xop, &ldx, &sx, st);
    if (s != HDC_OK) return s;
    if (use_tc(m)) {
        TcArgs a = {};
        a.Xq = Xop; a.N = N; a.F = m->Fk; a.ldx = (int)ldx; a.Bq = m->Bq; a.ldb = m->ldb; a.Dk = m->Dk; a.enc = m->enc;
        a.sx = sx; a.sb = m->b_scale; a.H = H; a.scores = scores; a.W = m->W;
        if (tc_supported(a)) return cu(timed_tc(a, st));
    }
    return cu(timed_simt(Xop, ldx, N, m->Fk, m->Bq, m->ldb, m->Dk, m->enc, sx, m->b_scale, H, m->W, scores,
                                 st));
}

hdc_status hdc_hamming_argmin(const uint32_t *Q, const uint32_t *Cls, int64_t N, int32_t C, int32_t D,
                              const hdc_approx_config *cfg, int32_t *labels, int32_t *dists, hdc_stream_t stream)
{
    Perf p;
    if (N < 0 || C <= 0 || D <= 0) return HDC_ERR_INVALID_ARG;
    if (cfg && (cfg->struct_size < sizeof(hdc_approx_config) || !perf_of(D, cfg, &p))) return HDC_ERR_INVALID_ARG;
    if (N == 0) return HDC_OK;
    if (!Q || !Cls || !labels || !aligned(Q, 16) || !aligned(Cls, 16)) return HDC_ERR_INVALID_ARG;
    const bool perforated = cfg && !(p.s0 == 0 && p.e0 == D && p.stride == 1);
    return cu(launch_similarity(Q, N, Cls, C, words_for(D), 1, D, perforated ? &p : nullptr, nullptr, nullptr,
                                labels, dists, nullptr, (cudaStream_t)stream));
}

hdc_status hdc_hamming_argmin_workspace_bytes(int32_t C, int32_t D, size_t *bytes)
{
    if (!bytes || C <= 0 || D <= 0) return HDC_ERR_INVALID_ARG;
    *bytes = align_up(class_sign_bytes(C, words_for(D)), kAlign);
    return HDC_OK;
}

hdc_status hdc_hamming_argmin_ws(const uint32_t *Q, const uint32_t *Cls, int64_t N, int32_t C, int32_t D,
                                 const hdc_approx_config *cfg, int32_t *labels, int32_t *dists, void *ws,
                                 size_t ws_bytes, hdc_stream_t stream)
{
    Perf p;
    if (N < 0 || C <= 0 || D <= 0) return HDC_ERR_INVALID_ARG;
    if (cfg && (cfg->struct_size < sizeof(hdc_approx_config) || !perf_of(D, cfg, &p))) return HDC_ERR_INVALID_ARG;
    const int W = words_for(D);
    const size_t need = class_sign_bytes(C, W);
    if (need && (!ws || ws_bytes < need || !aligned(ws, kAlign))) return HDC_ERR_WORKSPACE;
    if (N == 0) return HDC_OK;
    if (!Q || !Cls || !labels || !aligned(Q, 16) || !aligned(Cls, 16)) return HDC_ERR_INVALID_ARG;
    const bool perforated = cfg && !(p.s0 == 0 && p.e0 == D && p.stride == 1);
    const cudaStream_t st = (cudaStream_t)stream;
    if (!need)
        return cu(launch_similarity(Q, N, Cls, C, W, 1, D, perforated ? &p : nullptr, nullptr, nullptr, labels, dists,
                                    nullptr, st));
    // the classes once into ws (zero past D; the query bytes are zero
    // outside the kept dims), then the tensor-core route streams them
    uint8_t *signs = (uint8_t *)ws;
    hdc_status s = cu(launch_class_sign(Cls, C, W, D, (C + 15) / 16 * 16, hamming_packed_ldcs(W), signs, st));
    if (s != HDC_OK) return s;
    return cu(launch_hamming_packed(Q, N, Cls, C, W, D, perforated ? p.s0 : 0, perforated ? p.e0 : D,
                                    perforated ? p.stride : 1, labels, dists, st, signs));
}

namespace {
// Training workspace: predictions, the class-grouped sample order, the
// counting-sort histogram / offsets / first work item per group / cursors,
// the byte-lane bit counts of every counting item (32 bytes per item and
// word), and for 33..256 classes the class hypervectors expanded to bytes.
struct TrainLayout {
    size_t pred, perm, hist, offsets, items, cursor, partial, signs, total;
};
TrainLayout train_layout(int64_t N, int D, int C)
{
    TrainLayout L;
    size_t off = 0;
    L.pred = off;    off = align_up(off + (size_t)N * 4, kAlign);
    // retraining groups a misclassified sample twice (true and predicted
    // class): 2N permutation entries over 2C groups
    L.perm = off;    off = align_up(off + (size_t)2 * N * 4, kAlign);
    // histogram and cursors adjacent: zeroed by one memset
    L.hist = off;    L.cursor = off + (size_t)2 * C * 4;
    off = align_up(off + (size_t)4 * C * 4, kAlign);
    L.offsets = off; off = align_up(off + (size_t)(2 * C + 1) * 4, kAlign);
    L.items = off;   off = align_up(off + (size_t)(2 * C + 1) * 4, kAlign);
    L.partial = off; off = align_up(off + (size_t)train_max_items(N, C) * words_for(D) * 32, kAlign);
    L.signs = off;   off = align_up(off + class_sign_bytes(C, words_for(D)), kAlign);
    L.total = off;
    return L;
}
}  // namespace

hdc_status hdc_train_workspace_bytes(int64_t N, int32_t D, int32_t C, size_t *bytes)
{
    if (!bytes || N < 0 || D <= 0 || C <= 0) return HDC_ERR_INVALID_ARG;
    if (N > kMaxTrainRows || C > kMaxTrainClasses) return HDC_ERR_UNSUPPORTED;
    *bytes = train_layout(N, D, C).total;
    return HDC_OK;
}

hdc_status hdc_train_epoch(const uint32_t *H, const int32_t *y, int64_t N, int32_t D, int32_t C, int32_t mode,
                           int32_t *acc, uint32_t *cls, int32_t *n_updates, void *ws, size_t ws_bytes,
                           hdc_stream_t stream)
{
    if (N < 0 || D <= 0 || C <= 0 || mode < 0 || mode > 2 || !acc || !cls || !aligned(cls, 16))
        return HDC_ERR_INVALID_ARG;
    if (N > 0 && (!H || !y || !aligned(H, 16))) return HDC_ERR_INVALID_ARG;
    if (N > kMaxTrainRows || C > kMaxTrainClasses) return HDC_ERR_UNSUPPORTED;
    const int W = words_for(D);
    cudaStream_t st = (cudaStream_t)stream;
    const TrainLayout L = train_layout(N, D, C);
    if (N > 0 && (!ws || ws_bytes < L.total || !aligned(ws, kAlign))) return HDC_ERR_WORKSPACE;
    char *w = (char *)ws;
    if (n_updates) {
        hdc_status s = cu(cudaMemsetAsync(n_updates, 0, sizeof(int32_t), st));
        if (s != HDC_OK) return s;
    }
    if (N == 0) {
        // no samples: a bundle or a delta of zero; an epoch leaves acc as it is
        if (mode != 1) {
            hdc_status s = cu(cudaMemsetAsync(acc, 0, (size_t)C * D * sizeof(int32_t), st));
            if (s != HDC_OK) return s;
        }
        return mode == 2 ? HDC_OK : cu(launch_binarise(acc, C, D, cls, W, st));
    }
    TrainScratch sc = {(int32_t *)(w + L.perm), (int32_t *)(w + L.hist), (int32_t *)(w + L.offsets),
                       (int32_t *)(w + L.items), (int32_t *)(w + L.cursor), (uint32_t *)(w + L.partial),
                       class_sign_bytes(C, W) ? (uint8_t *)(w + L.signs) : nullptr};
    // mode 2 (a shard's delta) leaves cls as the start-of-epoch classes
    return cu(launch_train_pass(H, W, y, N, D, C, mode, cls, (int32_t *)(w + L.pred), acc,
                                mode == 2 ? nullptr : cls, n_updates, sc, st));
}

hdc_status hdc_train_apply(const int32_t *delta, int32_t C, int32_t D, int32_t *acc, uint32_t *cls,
                           hdc_stream_t stream)
{
    if (C <= 0 || D <= 0 || !acc || !cls || !aligned(cls, 16)) return HDC_ERR_INVALID_ARG;
    return cu(launch_apply_binarise(delta, acc, C, D, cls, words_for(D), (cudaStream_t)stream));
}

hdc_status hdc_classify(const float *X, int64_t N, const hdc_model *m, int32_t *labels, int32_t *dists,
                        double *scores, void *ws, size_t ws_bytes, hdc_stream_t stream)
{
    if (N < 0 || !model_ok(m) || m->C <= 0 || !m->cls) return HDC_ERR_INVALID_ARG;
    if (N == 0) return HDC_OK;
    if (!X || !labels || (ws_bytes && !ws) || (ws && !aligned(ws, kAlign))) return HDC_ERR_INVALID_ARG;
    const WsLayout L = ws_layout(N, m);
    if (ws_bytes < L.total) return HDC_ERR_WORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    const int nb = m->class_bits;
    if (!float_query(m->flags) && use_tc(m) && m->Fk == m->F && !scores) {
        // binary classes on the tensor cores: the fused kernel quantises its
        // own query tiles from X (the quantised operand never reaches HBM),
        // staging them in the quantised-query region of the workspace
        TcArgs a = {};
        a.N = N; a.F = m->Fk; a.ldx = ld_for(m->enc, m->Fk); a.Bq = m->Bq; a.ldb = m->ldb; a.Dk = m->Dk;
        a.enc = m->enc; a.sb = m->b_scale; a.W = m->W;
        a.planes = m->cls; a.C = m->C; a.nb = nb; a.csum = m->cls_sum; a.cnorm = m->cls_norm;
        a.labels = labels; a.dists = dists;
        a.cls_sign = m->cls_sign; a.ldcs = m->ldcs;
        a.X = X; a.ldX = m->F; a.stage = (uint8_t *)ws + L.xq;
        if (tc_qin_ok(a) && tc_stage_bytes(a) <= (size_t)N * a.ldx * esize_for(m->enc)) return cu(timed_tc(a, st));
    }
    const void *Xop;
    int64_t ldx;
    const float *sx;
    hdc_status s = prepare_queries(X, N, m, (char *)ws, L, &Xop, &ldx, &sx, st);
    if (s != HDC_OK) return s;
    uint32_t *Hb = (uint32_t *)((char *)ws + L.h);
    if (float_query(m->flags)) {
        // float queries: BF16 projections (tensor-core encoder's projection
        // epilogue, or FFMA projections converted), then the cosine GEMM
        uint16_t *sp = (uint16_t *)((char *)ws + L.sp);
        float *qn = (float *)((char *)ws + L.qn);
        const int ldS = lds_for(m->Dk);
        bool done = false;
        if (use_tc(m) && m->C <= 128) {
            // encode and cosine fused: the BF16 projections stay on chip
            TcArgs f = {};
            f.Xq = Xop; f.N = N; f.F = m->Fk; f.ldx = (int)ldx; f.Bq = m->Bq; f.ldb = m->ldb; f.Dk = m->Dk;
            f.enc = m->enc; f.sx = sx; f.sb = m->b_scale; f.W = m->W; f.C = m->C; f.labels = labels;
            if (t_prof_start) cudaEventRecord(t_prof_start, st);
            const cudaError_t e = launch_tc_fcos(f, (const uint16_t *)m->cls, ldS, m->cls_norm, scores, st);
            if (t_prof_stop) cudaEventRecord(t_prof_stop, st);
            if (e != cudaErrorNotSupported) return cu(e);
        }
        if (use_tc(m)) {
            TcArgs e = {};
            e.Xq = Xop; e.N = N; e.F = m->Fk; e.ldx = (int)ldx; e.Bq = m->Bq; e.ldb = m->ldb; e.Dk = m->Dk;
            e.enc = m->enc; e.sx = sx; e.sb = m->b_scale; e.W = m->W; e.sproj = sp; e.ldS = ldS; e.qn = qn;
            if (tc_supported(e)) {
                s = cu(timed_tc(e, st));
                if (s != HDC_OK) return s;
                done = true;
            }
        }
        if (!done) {
            // FFMA projections carry the query row's scale too (a power of
            // two, common to the row: neither BF16 rounding nor the cosine
            // changes relative to the dropped-scale definition)
            float *sf = (float *)((char *)ws + L.sf);
            s = cu(timed_simt(Xop, ldx, N, m->Fk, m->Bq, m->ldb, m->Dk, m->enc, sx, m->b_scale, Hb, m->W, sf, st));
            if (s != HDC_OK) return s;
            s = cu(launch_proj_bf16(sf, N, m->Dk, sp, ldS, qn, st));
            if (s != HDC_OK) return s;
        }
        CosArgs c = {};
        c.q = sp; c.qn = qn; c.N = N; c.ldS = ldS; c.cv = (const uint16_t *)m->cls; c.cnorm = m->cls_norm;
        c.C = m->C; c.Cp = cpad_for(m->C); c.labels = labels; c.scores = scores;
        return cu(launch_tc_cosine(c, st));
    }
    bool encoded = false;
    if (use_tc(m)) {
        TcArgs a = {};
        a.Xq = Xop; a.N = N; a.F = m->Fk; a.ldx = (int)ldx; a.Bq = m->Bq; a.ldb = m->ldb; a.Dk = m->Dk; a.enc = m->enc;
        a.sx = sx; a.sb = m->b_scale; a.W = m->W;
        a.planes = m->cls; a.C = m->C; a.nb = nb; a.csum = m->cls_sum; a.cnorm = m->cls_norm;
        a.labels = labels; a.dists = dists; a.sims = scores;
        a.cls_sign = m->cls_sign; a.ldcs = m->ldcs;
        a.dacc = (int32_t *)((char *)ws + L.dacc);
        // binary classes: fully fused; otherwise tensor-core encode + K4
        if (tc_supported(a)) return cu(timed_tc(a, st));
        a.dacc = nullptr;
        TcArgs e = a;
        e.planes = nullptr; e.labels = nullptr; e.dists = nullptr; e.sims = nullptr; e.H = Hb;
        if (tc_supported(e)) {
            s = cu(timed_tc(e, st));
            if (s != HDC_OK) return s;
            encoded = true;
        }
    }
    if (!encoded) {
        s = cu(timed_simt(Xop, ldx, N, m->Fk, m->Bq, m->ldb, m->Dk, m->enc, sx, m->b_scale, Hb, m->W,
                                  nullptr, st));
        if (s != HDC_OK) return s;
    }
    if (classify_sign_bytes(m)) {   // 129..256 binary classes: the classes expanded once, then the tensor cores
        uint8_t *signs = (uint8_t *)ws + L.csign;
        s = cu(launch_class_sign(m->cls, m->C, m->W, m->Dk, (m->C + 15) / 16 * 16, hamming_packed_ldcs(m->W), signs,
                                 st));
        if (s != HDC_OK) return s;
        return cu(launch_hamming_packed(Hb, N, m->cls, m->C, m->W, m->Dk, 0, m->Dk, 1, labels, dists, st, signs));
    }
    return cu(launch_similarity(Hb, N, m->cls, m->C, m->W, nb, m->Dk, nullptr, m->cls_sum, m->cls_norm, labels,
                                dists, scores, st));
}

hdc_status hdc_stream_status(hdc_stream_t stream)
{
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaStreamSynchronize(st) != cudaSuccess) return HDC_ERR_CUDA;
    int status = 0, qstatus = 0;
    if (tc_read_status(st, &status) != cudaSuccess) return HDC_ERR_CUDA;
    if (quant_read_status(st, &qstatus) != cudaSuccess) return HDC_ERR_CUDA;
    if (!status) status = qstatus;
    if (status == 1) return HDC_ERR_TIMEOUT;
    if (status != 0) return HDC_ERR_DEVICE;
    return HDC_OK;
}

hdc_status hdc_selftest_wait(uint32_t limit_us, hdc_stream_t stream)
{
    if (limit_us < 1 || limit_us > 2000000) return HDC_ERR_INVALID_ARG;
    return cu(launch_wait_selftest((unsigned long long)limit_us * 1000ull, (cudaStream_t)stream));
}

void hdc_profile_events(void *start, void *stop)
{
    t_prof_start = (cudaEvent_t)start;
    t_prof_stop = (cudaEvent_t)stop;
}

const char *hdc_status_string(hdc_status s)
{
    switch (s) {
    case HDC_OK: return "ok";
    case HDC_ERR_INVALID_ARG: return "invalid argument";
    case HDC_ERR_UNSUPPORTED: return "unsupported configuration";
    case HDC_ERR_WORKSPACE: return "buffer or workspace too small";
    case HDC_ERR_CUDA: return "CUDA error";
    case HDC_ERR_TIMEOUT: return "device wait timed out";
    case HDC_ERR_DEVICE: return "device-side check failed";
    }
    return "unknown status";
}

}  // extern "C"
