// Host side of the tensor-core encoder: TMA tensor maps, support checks,
// grid sizing and dispatch to the per-encoding translation units.
#include <cudaTypedefs.h>

#include <mutex>

#include "tc_fcos16.cuh"

namespace hdc {
namespace {

PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ptr);
    });
    return fn;
}

// 2-D map over a row-major [rows x F] operand with row stride ld; box = 128 bytes of K by
// box_rows rows, 128-byte swizzle, zero fill outside the tensor.
bool make_map(CUtensorMap *m, const void *base, int enc, int F, int ld, int64_t rows, int box_rows)
{
    auto fn = encode_fn();
    if (!fn) return false;
    const int es = enc == HDC_ENC_BF16 ? 2 : 1;
    // the map spans the padded stride (zeros past F): boxes never leave the
    // tensor, which measured faster than letting TMA zero-fill the K tail
    (void)F;
    cuuint64_t dims[2] = {(cuuint64_t)ld, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ld * es};
    cuuint32_t box[2] = {(cuuint32_t)(tc::BKB / es), (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(m, enc == HDC_ENC_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_UINT8, 2,
                    const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// Map over the binary class words (C rows x W uint32): box = 8 words (one
// 256-dim tile) x C rows, no swizzle, zeros past W.
bool make_cls_map(CUtensorMap *m, const uint32_t *planes, int W, int C)
{
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)W, (cuuint64_t)C};
    cuuint64_t strides[1] = {(cuuint64_t)W * 4};
    cuuint32_t box[2] = {8, (cuuint32_t)C};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_UINT32, 2, const_cast<uint32_t *>(planes), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// Map over the E4M3 +-1 class bytes (Cp rows x ldcs bytes): box = one
// 128-byte K atom x Cp rows, 128-byte swizzle (the MMA operand layout).
bool make_sign_map(CUtensorMap *m, const uint8_t *signs, int ldcs, int Cp)
{
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)ldcs, (cuuint64_t)Cp};
    cuuint64_t strides[1] = {(cuuint64_t)ldcs};
    cuuint32_t box[2] = {128, (cuuint32_t)Cp};
    cuuint32_t estr[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<uint8_t *>(signs), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int sm_count()
{
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    return n;
}

}  // namespace

// The class-byte map for the other tensor-core translation units.
bool make_class_sign_map(CUtensorMap *m, const uint8_t *signs, int ldcs, int Cp)
{
    return make_sign_map(m, signs, ldcs, Cp);
}

bool tc_supported(const TcArgs &a)
{
    if (a.enc != HDC_ENC_BF16 && a.enc != HDC_ENC_FP8_E4M3) return false;
    const int es = a.enc == HDC_ENC_BF16 ? 2 : 1;
    if (a.F <= 0 || a.ldx != a.ldb || a.ldx < a.F || (a.ldx * es) % 16 != 0) return false;
    if (a.N <= 0 || a.N > 0x7fffffffLL - tc::BM || a.Dk <= 0 || a.W != words_for(a.Dk)) return false;
    // fused classify: binary class hypervectors, up to 128 classes
    if (a.planes && (a.C <= 0 || a.C > 128 || a.nb != 1)) return false;
    if (!a.planes && !a.H && !a.sproj) return false;
    if (a.sproj && (a.planes || !a.qn || a.ldS % 64 != 0 || a.ldS < a.Dk)) return false;
    if (!encode_fn()) return false;
    return true;
}

namespace {
unsigned tc_grid(int64_t N, int sms)
{
    const int64_t m_tiles = (N + tc::BM - 1) / tc::BM;
    return (unsigned)(m_tiles < sms ? m_tiles : sms);
}
}  // namespace

// The fused classify routes that can quantise their own query tiles: the
// popcount epilogue with one or two warpgroups (up to 32 classes) and the
// tensor-core Hamming kernel (33..112 classes with their E4M3 signs).
bool tc_qin_route(const TcArgs &a)
{
    return a.C <= 32 || (a.cls_sign && a.C <= tc::H_CMAX);
}

bool tc_qin_ok(const TcArgs &a)
{
    if (!a.X || !a.stage || !a.planes || a.C <= 0 || !tc_qin_route(a) || a.nb != 1 || a.H || a.sproj || a.scores ||
        a.sims)
        return false;
    if (!tc_supported(a) || a.ldx > tc::QIN_MAX_LD || a.F % 4 != 0 || a.ldX % 4 != 0 || a.ldX < a.F ||
        (uintptr_t)a.X % 16 != 0 || (uintptr_t)a.stage % 16 != 0)
        return false;
    const int sms = sm_count();
    if (sms <= 0) return false;
    // The quantiser warps keep a few rows in flight each, so a tile's FP32
    // rows take about as long as 0.15 * F of its 128-byte MMA stages.  With
    // fewer stages per tile they set the pace, and the row-quantiser pass
    // (at the HBM rate) plus the fused kernel is faster.  Measured on GB300
    // (1,048,576 queries, F = 784, E4M3, two builds alternated): 140 stages
    // per tile 3.54 vs 3.59 ms, 280 stages 6.26 vs 6.58 ms, 70 stages 2.82
    // vs 2.11 ms.
    const int es = a.enc == HDC_ENC_BF16 ? 2 : 1;
    const int tile_n = a.C > 32 ? tc::HBN : tc::BN;
    const int64_t stages = (int64_t)((a.Dk + tile_n - 1) / tile_n) * ((a.ldx * es + tc::BKB - 1) / tc::BKB);
    if (20 * stages < (int64_t)3 * a.F) return false;
    // two staged tiles per CTA fit in the N rows of the quantised operand
    return a.N >= (int64_t)2 * tc_grid(a.N, sms) * tc::BM;
}

size_t tc_stage_bytes(const TcArgs &a)
{
    const int sms = sm_count();
    if (sms <= 0) return 0;
    return (size_t)2 * tc_grid(a.N, sms) * tc::BM * a.ldx * (a.enc == HDC_ENC_BF16 ? 2 : 1);
}

cudaError_t launch_tc_encode(const TcArgs &a, cudaStream_t st)
{
    CUtensorMap ma, mb;
    const bool qin = a.X != nullptr;
    if (qin && !tc_qin_ok(a)) return cudaErrorNotSupported;
    const int sms = sm_count();
    if (sms <= 0) return cudaErrorNoDevice;
    unsigned grid = tc_grid(a.N, sms);
    // QIN: the A operand is the CTAs' staged tiles (2 per CTA)
    if (!(qin ? make_map(&ma, a.stage, a.enc, a.F, a.ldx, (int64_t)2 * grid * tc::BM, tc::BM)
              : make_map(&ma, a.Xq, a.enc, a.F, a.ldx, a.N, tc::BM)) ||
        !make_map(&mb, a.Bq, a.enc, a.F, a.ldb, a.Dk, tc::BN))
        return cudaErrorInvalidValue;
    tc::Params p;
    p.N = a.N;
    p.Dk = a.Dk;
    // K blocks of 128 bytes over the padded row (zeros past F); the last
    // block issues only the 32-byte K steps that reach into [0, F)
    const int es = a.enc == HDC_ENC_BF16 ? 2 : 1;
    p.num_kb = (a.ldx * es + tc::BKB - 1) / tc::BKB;
    p.last_k = (a.F * es - (p.num_kb - 1) * tc::BKB + 31) / 32;
    if (p.last_k < 1 || p.last_k > tc::BKB / 32) p.last_k = tc::BKB / 32;
    p.W = a.W;
    p.sx = a.sx;
    p.sb = a.sb;
    p.H = a.H;
    p.scores = a.scores;
    p.planes = a.planes;
    p.C = a.C;
    p.labels = a.labels;
    p.dists = a.dists;
    p.sproj = a.sproj;
    p.ldS = a.ldS;
    p.qn = a.qn;
    if (qin) {
        p.X = a.X;
        p.ldX = a.ldX;
        p.F = a.F;
        p.ld = a.ldx;
        p.stage = a.stage;
    }
    const bool classify = a.planes != nullptr;
    if (classify && a.cls_sign && a.nb == 1 && a.C > 32 && a.C <= tc::H_CMAX) {
        // binary classes, 33..112 of them: Hamming distances on the tensor
        // cores (a second MMA of the sign tile against the class signs); up
        // to 32 the 256-dim tiles with the popcount epilogue measured faster
        // (F 617, D 2,048, 26 classes: 1.22 vs 1.59 ms per 2^20 queries)
        CUtensorMap mb2, ms;
        const int Cp = (a.C + 15) / 16 * 16;
        if (!make_map(&mb2, a.Bq, a.enc, a.F, a.ldb, a.Dk, tc::HBN) || !make_sign_map(&ms, a.cls_sign, a.ldcs, Cp))
            return cudaErrorInvalidValue;
        tc::HParams h;
        h.N = a.N;
        h.Dk = a.Dk;
        h.num_kb = p.num_kb;
        h.nt = (a.Dk + tc::HBN - 1) / tc::HBN;
        h.C = a.C;
        h.Cp = Cp;
        h.labels = a.labels;
        h.dists = a.dists;
        if (qin) {
            h.X = a.X;
            h.ldX = a.ldX;
            h.F = a.F;
            h.ld = a.ldx;
            h.stage = a.stage;
        }
        if (a.ldcs < h.nt * tc::HBN + 64) return cudaErrorInvalidValue;
        if (a.enc == HDC_ENC_BF16) return tc::launch_hamming_bf16(ma, mb2, ms, h, grid, st);
        return tc::launch_hamming_fp8(ma, mb2, ms, h, grid, st);
    }
    CUtensorMap mc = mb;  // unused by encode-only launches
    if (classify && !make_cls_map(&mc, a.planes, a.W, a.C)) return cudaErrorInvalidValue;
    // few query tiles: split each tile's dim tiles over CTAs so that the
    // batch fills the SMs (non-empty ranges only); partial distances meet
    // in the zero-filled scratch
    const int64_t m_tiles = (a.N + tc::BM - 1) / tc::BM;
    const int n_tiles = (a.Dk + tc::BN - 1) / tc::BN;
    unsigned g = grid;
    if (classify && !qin && a.dacc && m_tiles < sms && m_tiles <= TC_SPLIT_MAX_TILES) {
        int ns = (int)(sms / m_tiles);
        if (ns > n_tiles) ns = n_tiles;
        const int per = (n_tiles + ns - 1) / ns;
        ns = (n_tiles + per - 1) / per;
        if (ns > 1) {
            p.nsplit = ns;
            p.dacc = a.dacc;
            p.tile_done = reinterpret_cast<unsigned *>(reinterpret_cast<char *>(a.dacc) +
                                                       (size_t)a.N * a.C * 4);
            const cudaError_t e = cudaMemsetAsync(a.dacc, 0, (size_t)a.N * a.C * 4 + (size_t)m_tiles * 4, st);
            if (e != cudaSuccess) return e;
            const int64_t units = m_tiles * ns;
            g = (unsigned)(units < sms ? units : sms);
        }
    }
    grid = g;
    if (a.enc == HDC_ENC_BF16) return tc::launch_bf16(ma, mb, mc, p, grid, classify, st);
    return tc::launch_fp8(ma, mb, mc, p, grid, classify, st);
}

cudaError_t launch_tc_fcos(const TcArgs &a, const uint16_t *cv, int ldS, const double *cnorm, double *scores,
                          cudaStream_t st)
{
    if (a.C <= 0 || a.C > tc::FC_CMAX || a.N <= 0 || a.N > 0x7fffffffLL - tc::BM || !cv || !cnorm || !a.labels ||
        ldS % 64 != 0 || ldS < a.Dk)
        return cudaErrorNotSupported;
    // the encoder's operand rules (as tc_supported)
    if (a.enc != HDC_ENC_BF16 && a.enc != HDC_ENC_FP8_E4M3) return cudaErrorNotSupported;
    if (a.F <= 0 || a.ldx != a.ldb || a.ldx < a.F || (a.ldx * (a.enc == HDC_ENC_BF16 ? 2 : 1)) % 16 != 0 ||
        a.Dk <= 0)
        return cudaErrorNotSupported;
    auto fn = encode_fn();
    if (!fn) return cudaErrorNotSupported;
    const int Cp = (a.C + 15) / 16 * 16;
    // up to 16 classes: 256-dim encode tiles with the cosine partials in the
    // tile's own accumulator (tc_fcos16.cuh); more: 192-dim tiles and a
    // cosine accumulator of its own (tc_fcos.cuh)
    const bool small_c = Cp == tc::F16_CP;
    CUtensorMap ma, mb, mv;
    if (!make_map(&ma, a.Xq, a.enc, a.F, a.ldx, a.N, tc::BM) ||
        !make_map(&mb, a.Bq, a.enc, a.F, a.ldb, a.Dk, small_c ? tc::BN : tc::HBN))
        return cudaErrorInvalidValue;
    {
        cuuint64_t dims[2] = {(cuuint64_t)ldS, (cuuint64_t)Cp};
        cuuint64_t strides[1] = {(cuuint64_t)ldS * 2};
        cuuint32_t box[2] = {64, (cuuint32_t)Cp};
        cuuint32_t estr[2] = {1, 1};
        if (fn(&mv, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<uint16_t *>(cv), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    tc::FCParams p;
    p.N = a.N;
    p.Dk = a.Dk;
    const int es = a.enc == HDC_ENC_BF16 ? 2 : 1;
    p.num_kb = (a.ldx * es + tc::BKB - 1) / tc::BKB;
    p.nt = small_c ? (a.Dk + tc::BN - 1) / tc::BN : (a.Dk + tc::HBN - 1) / tc::HBN;
    p.C = a.C;
    p.Cp = Cp;
    p.sb = a.sb;
    p.cnorm = cnorm;
    p.labels = a.labels;
    p.scores = scores;
    const int sms = sm_count();
    if (sms <= 0) return cudaErrorNoDevice;
    const int64_t m_tiles = (a.N + tc::BM - 1) / tc::BM;
    const unsigned grid = (unsigned)(m_tiles < sms ? m_tiles : sms);
    if (small_c) {
        CUtensorMap ms = mv;   // unread without scales (BF16)
        if (a.sb) {            // the Dk base-row scales as one row, boxes of one tile, zero past Dk
            cuuint64_t dims[2] = {(cuuint64_t)a.Dk, 1};
            cuuint64_t strides[1] = {((cuuint64_t)a.Dk * 4 + 15) / 16 * 16};
            cuuint32_t box[2] = {(cuuint32_t)tc::BN, 1};
            cuuint32_t estr[2] = {1, 1};
            if (fn(&ms, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(a.sb), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
                return cudaErrorInvalidValue;
        }
        if (a.enc == HDC_ENC_BF16) return tc::launch_fcos16_bf16(ma, mb, mv, ms, p, grid, st);
        return tc::launch_fcos16_fp8(ma, mb, mv, ms, p, grid, st);
    }
    if (a.enc == HDC_ENC_BF16) return tc::launch_fcos_bf16(ma, mb, mv, p, grid, st);
    return tc::launch_fcos_fp8(ma, mb, mv, p, grid, st);
}

cudaError_t tc_read_status(cudaStream_t st, int *status)
{
    int a = 0, b = 0, c = 0, x = 0;
    cudaError_t e = tc::status_bf16(st, &a);
    if (e == cudaSuccess) e = tc::status_fp8(st, &b);
    if (e == cudaSuccess) e = tc_cosine_read_status(st, &c);
    if (e == cudaSuccess) e = tc_aux_read_status(st, &x);
    *status = a ? a : b ? b : c ? c : x;
    return e;
}

}  // namespace hdc
