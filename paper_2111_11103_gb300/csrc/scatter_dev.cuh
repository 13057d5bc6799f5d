// Device side of the pipelined scatter (Sec. 3.3.2 update of the rows of P,
// Eqs. sum / mul / maxsum and their weighted forms), shared by the
// stream-ordered scatter kernel (scatter.cu) and the persistent work-queue
// kernel (queue.cu): decoding of the stored probabilities, the per-pixel row
// / weight / scale lookup, the run-building warp walks and the drain of a
// warp's entries into P.  See scatter.cu for the design.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "lf_internal.cuh"
#include "ptx.cuh"

namespace lf {
namespace sdev {


constexpr int kConsumerWarps = 8;   // 32 pixels each
constexpr int kTile = 32 * kConsumerWarps;  // pixels per tile
constexpr int kThreads = 32 * (1 + kConsumerWarps);
constexpr int kUnroll = 4;          // pixels per software-pipelined step
constexpr int kMaxFactors = 4;      // probabilities multiplied before one log2 (a power of two)
static_assert((kMaxFactors & (kMaxFactors - 1)) == 0, "run splitting masks with kMaxFactors - 1");
constexpr uint64_t kWaitNs = 2000000000ull;
constexpr float kLn2 = 0.693147180559945309f;
constexpr unsigned kFull = 0xffffffffu;

template <int DT>
struct Elem {
    static constexpr int size = DT == SM_F32 ? 4 : (DT == SM_BF16 ? 2 : 1);
};

// Four consecutive classes starting at element index e (a multiple of 4).
template <int DT, bool SMEM>
__device__ __forceinline__ float4 load_quad(const uint8_t *base, int e)
{
    if (DT == SM_F32) {
        const float4 *p = reinterpret_cast<const float4 *>(base + e * 4);
        return SMEM ? *p : __ldcs(p);
    } else if (DT == SM_BF16) {
        const uint2 *p = reinterpret_cast<const uint2 *>(base + e * 2);
        const uint2 u = SMEM ? *p : __ldcs(p);
        return make_float4(__uint_as_float(u.x << 16), __uint_as_float(u.x & 0xffff0000u),
                           __uint_as_float(u.y << 16), __uint_as_float(u.y & 0xffff0000u));
    } else {
        const unsigned int *p = reinterpret_cast<const unsigned int *>(base + e);
        const unsigned int u = SMEM ? *p : __ldcs(p);
        __half2_raw lo = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(u & 0xffffu), __NV_E4M3);
        __half2_raw hi = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(u >> 16), __NV_E4M3);
        const float2 a = __half22float2(*reinterpret_cast<__half2 *>(&lo));
        const float2 b = __half22float2(*reinterpret_cast<__half2 *>(&hi));
        return make_float4(a.x, a.y, b.x, b.y);
    }
}

__device__ __forceinline__ float4 scale4(float4 v, float s)
{
    return make_float4(__fmul_rn(v.x, s), __fmul_rn(v.y, s), __fmul_rn(v.z, s), __fmul_rn(v.w, s));
}

struct ScatterArgs {
    const uint8_t *probs;
    const float *scale;
    unsigned long long *keys;  // face mode: z-buffer keys (read and re-armed)
    const int32_t *ids_in;     // otherwise: row map (16-byte aligned)
    int32_t *ids_out;          // optional row map output
    int64_t total_px, npix;
    int c;
    const uint32_t *fcnt;      // per-frame row histogram (image weights) or null
    float alpha;               // image-weight mix (1: w^(I))
    const float *wpix;         // explicit per-pixel weights (replace the histogram), or null
    int64_t n_x;
    float *acc;
    uint32_t *cnt;
    int32_t *err;
    bool scale_bulk;           // per-pixel scales copied with the tile
    uint64_t wait_ns;          // limit of every barrier wait
    int skip_it;               // test hook: the producer skips this pipeline step (-1: never)
};

// Stage layout: probabilities | keys (8 B/px) or row ids (4 B/px) | scales.
struct StageLayout {
    uint32_t probs_bytes, meta_bytes, scale_bytes, stride;
};

template <int DT>
__host__ __device__ __forceinline__ StageLayout stage_layout(const ScatterArgs &a)
{
    StageLayout L;
    L.probs_bytes = (uint32_t)kTile * a.c * Elem<DT>::size;
    L.meta_bytes = kTile * (a.keys ? 8u : 4u);
    L.scale_bytes = (DT != SM_F32 && a.scale_bulk) ? kTile * 4u : 0u;
    L.stride = (L.probs_bytes + L.meta_bytes + L.scale_bytes + 127u) & ~127u;
    return L;
}

// Row, weight and scale of pixel p.  meta/sscale point at the stage's
// metadata (null for the ragged tile, which reads global memory); i is the
// pixel's index within its tile.
template <int DT, bool IMAGE>
__device__ __forceinline__ void pixel_info(const ScatterArgs &a, int64_t p, int i, const uint8_t *meta, const float *sscale,
                                           int &row, float &w, float &sc)
{
    row = -1;
    w = 1.0f;
    sc = 1.0f;
    if (p >= a.total_px) return;
    if (a.keys) {
        const unsigned long long key =
            meta ? reinterpret_cast<const unsigned long long *>(meta)[i] : a.keys[p];
        a.keys[p] = kEmptyKey;
        row = (key == kEmptyKey) ? -1 : (int)(unsigned int)key;
    } else {
        row = meta ? reinterpret_cast<const int32_t *>(meta)[i] : a.ids_in[p];
    }
    if (a.ids_out) a.ids_out[p] = row;
    if (row >= a.n_x) {
        atomicCAS(a.err, 0, (int32_t)kErrRowRange);
        row = -1;
    }
    if (IMAGE && row >= 0) w = a.wpix ? a.wpix[p] : image_weight(a.alpha, a.fcnt[frame_of(p, a.npix) * a.n_x + row]);
    if (DT != SM_F32) sc = sscale ? sscale[i] : a.scale[p];
}

// Running state of one lane's four classes over the current run.
struct Run {
    float4 s;     // sum of w * phi (log-sum: natural logarithms)
    float4 prod;  // log-sum: product of the clamped probabilities not yet logged
    int nf;       // factors in prod
};

__device__ __forceinline__ void fold_logs(Run &r, float w)
{
    const float wl = w * kLn2;
    r.s.x = fmaf(lg2_ftz(r.prod.x), wl, r.s.x);
    r.s.y = fmaf(lg2_ftz(r.prod.y), wl, r.s.y);
    r.s.z = fmaf(lg2_ftz(r.prod.z), wl, r.s.z);
    r.s.w = fmaf(lg2_ftz(r.prod.w), wl, r.s.w);
    r.prod = make_float4(1.f, 1.f, 1.f, 1.f);
    r.nf = 0;
}

// Adds a finished run into its row: the group's lanes write one contiguous
// row (16 bytes each), the first lane adds the run length to the count.
template <int RULE>
__device__ __forceinline__ void flush(const ScatterArgs &a, float *accq, int cur, float w, Run &r, uint32_t n, int q)
{
    if (cur < 0) return;
    if (RULE == SM_RULE_LOGSUM && r.nf > 0) fold_logs(r, w);
    const uint64_t keep = l2_evict_last();
    red_add_v4(accq + (int64_t)cur * a.c, r.s, keep);
    if (q == 0) red_add_u32(a.cnt + cur, n, keep);
}

// phi(p) of one pixel added into the run (weight wk); pix points at the
// pixel's first element (max-sum and vote scan the whole pixel).
template <int RULE, int DT, bool SMEM>
__device__ __forceinline__ void accumulate(Run &r, float4 v, float wk, float sk, const uint8_t *pix, int q, int Q)
{
    if (RULE == SM_RULE_SUM) {
        r.s.x = fmaf(wk, v.x, r.s.x);
        r.s.y = fmaf(wk, v.y, r.s.y);
        r.s.z = fmaf(wk, v.z, r.s.z);
        r.s.w = fmaf(wk, v.w, r.s.w);
    } else if (RULE == SM_RULE_LOGSUM) {
        r.prod.x *= fmaxf(v.x, kPMin);
        r.prod.y *= fmaxf(v.y, kPMin);
        r.prod.z *= fmaxf(v.z, kPMin);
        r.prod.w *= fmaxf(v.w, kPMin);
        if (++r.nf == kMaxFactors) fold_logs(r, wk);
    } else {
        // maximum (and first arg max) of the whole pixel, scanned in class order
        float m = -INFINITY;
        int am = 0;
        for (int j = 0; j < Q; ++j) {
            float4 u = load_quad<DT, SMEM>(pix, 4 * j);
            if (DT != SM_F32) u = scale4(u, sk);
            if (j == 0 || u.x > m) { m = u.x; am = 4 * j; }
            if (u.y > m) { m = u.y; am = 4 * j + 1; }
            if (u.z > m) { m = u.z; am = 4 * j + 2; }
            if (u.w > m) { m = u.w; am = 4 * j + 3; }
        }
        if (RULE == SM_RULE_MAXSUM) {
            if (v.x == m) r.s.x = fmaf(wk, v.x, r.s.x);
            if (v.y == m) r.s.y = fmaf(wk, v.y, r.s.y);
            if (v.z == m) r.s.z = fmaf(wk, v.z, r.s.z);
            if (v.w == m) r.s.w = fmaf(wk, v.w, r.s.w);
        } else {
            const int d = am - 4 * q;
            if (d == 0) r.s.x += wk;
            if (d == 1) r.s.y += wk;
            if (d == 2) r.s.z += wk;
            if (d == 3) r.s.w += wk;
        }
    }
}

// One warp's 32 pixels of a tile.  base points at the tile's first element
// (shared memory stage, or global memory for the ragged last tile); px0 is
// the warp's first pixel within the tile; row/w/sc belong to pixel px0+lane.
// A run is cut where the row or the pixel weight changes.
template <int RULE, int DT, bool SMEM, bool IMAGE>
__device__ __forceinline__ void warp_tile(const ScatterArgs &a, const uint8_t *base, int px0, int lane, int row, float w,
                                          float sc)
{
    constexpr int ES = Elem<DT>::size;
    const int Q = a.c >> 2;
    const int G = 32 / Q;
    const int g = lane / Q, q = lane - g * Q;
    const bool active = g < G;
    const int start = active ? (32 * g) / G : 0;
    const int len = active ? (32 * (g + 1)) / G - start : 0;
    const int iters = (32 + G - 1) / G;
    const int pstride = a.c * ES;  // bytes per pixel
    const uint8_t *pb = base + (px0 + start) * pstride;  // this group's first pixel
    float *accq = a.acc + 4 * q;
    Run run{make_float4(0.f, 0.f, 0.f, 0.f), make_float4(1.f, 1.f, 1.f, 1.f), 0};
    int cur = -1;
    float curw = 1.0f;
    uint32_t n = 0;
    for (int i0 = 0; i0 < iters; i0 += kUnroll) {
        int r[kUnroll];
        float wv[kUnroll], sv[kUnroll];
        float4 v[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const int k = (start + i0 + u) & 31;
            r[u] = __shfl_sync(kFull, row, k);
            wv[u] = IMAGE ? __shfl_sync(kFull, w, k) : 1.0f;
            sv[u] = (DT != SM_F32) ? __shfl_sync(kFull, sc, k) : 1.0f;
            if (i0 + u >= len) r[u] = -2;  // past this group's run (or inactive lane)
        }
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            v[u] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (r[u] >= 0) {
                v[u] = load_quad<DT, SMEM>(pb + (i0 + u) * pstride, 4 * q);
                if (DT != SM_F32) v[u] = scale4(v[u], sv[u]);
            }
        }
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            if (r[u] == -2) continue;
            if (r[u] != cur || (IMAGE && wv[u] != curw)) {
                flush<RULE>(a, accq, cur, curw, run, n, q);
                cur = r[u];
                curw = wv[u];
                run.s = make_float4(0.f, 0.f, 0.f, 0.f);
                run.prod = make_float4(1.f, 1.f, 1.f, 1.f);
                run.nf = 0;
                n = 0;
            }
            if (r[u] < 0) continue;
            accumulate<RULE, DT, SMEM>(run, v[u], wv[u], sv[u], pb + (i0 + u) * pstride, q, Q);
            ++n;
        }
    }
    if (active) flush<RULE>(a, accq, cur, curw, run, n, q);
}

// Entries of one warp tile, for a compile-time class count C.  An entry is a
// run of consecutive pixels of one group with the same row and weight (log-
// sum: at most kMaxFactors pixels, so the product of its clamped
// probabilities cannot underflow).  Its C values (sums of phi, or the
// products) sit in a per-warp array of 32 entries in shared memory; row,
// length and weight in EntryMeta.  A tile has at most 32 entries (one per
// pixel), so the array never overflows.
struct EntryMeta {
    int row[32];
    uint32_t n[32];
    float w[32];
};

template <int C, int DT>
struct EntryLayout {
    // with FP32 storage a warp's 32 pixels of the stage are exactly 32
    // entries: once they are in registers the entries overwrite them
    static constexpr bool kInStage = Elem<DT>::size == 4;
    static constexpr uint32_t kMetaBytes = kConsumerWarps * sizeof(EntryMeta);
    static constexpr uint32_t kQueueBytes = kInStage ? 0u : kConsumerWarps * 32u * C * 4u;
    static constexpr uint32_t bytes = C != 0 ? (kMetaBytes + kQueueBytes + 127u) & ~127u : 0u;
};

// Adds the warp's entries into their rows of P (16-byte reductions, L2
// evict-last: the rows a trajectory keeps revisiting stay in L2 while the
// prediction stream passes through) and their lengths into the observation
// counts.  The whole warp takes part, 32 quads per instruction.
// PAIRED: two quads per lane and iteration, both loaded before either is
// used, so that their shared-memory and logarithm latencies overlap (measured
// faster for FP32 storage, slower for FP8, where the one-quad loop is kept).
template <int C, int RULE, bool IMAGE, bool PAIRED>
__device__ __forceinline__ void drain(const ScatterArgs &a, const float4 *queue, const EntryMeta &meta, int E, int lane)
{
    constexpr int Q = C / 4;
    const uint64_t keep = l2_evict_last();
    auto one = [&](int k, int r, float4 v, float we) {
        if ((uint64_t)(int64_t)r >= (uint64_t)a.n_x) {  // never for a consistent layout: latch, skip
            atomicCAS(a.err, 0, (int32_t)kErrRowRange);
            return;
        }
        if (RULE == SM_RULE_LOGSUM) {
            // sum_k w log p_k = w ln 2 log2 prod_k p_k
            const float wl = (IMAGE ? we : 1.0f) * kLn2;
            v = make_float4(lg2_ftz(v.x) * wl, lg2_ftz(v.y) * wl, lg2_ftz(v.z) * wl, lg2_ftz(v.w) * wl);
        } else if (IMAGE) {
            v = make_float4(v.x * we, v.y * we, v.z * we, v.w * we);
        }
        red_add_v4(a.acc + (int64_t)r * C + 4 * (k - (k / Q) * Q), v, keep);
    };
    const int n = E * Q;
    if (PAIRED) {
        for (int k = lane; k < n; k += 64) {
            const int k2 = k + 32;
            const bool two = k2 < n;
            const int e = k / Q, e2 = two ? k2 / Q : e;
            const int r = meta.row[e], r2 = meta.row[e2];
            const float we = IMAGE ? meta.w[e] : 1.0f, we2 = IMAGE ? meta.w[e2] : 1.0f;
            const float4 v = queue[k];
            const float4 v2 = two ? queue[k2] : v;
            one(k, r, v, we);
            if (two) one(k2, r2, v2, we2);
        }
    } else {
        for (int k = lane; k < n; k += 32) {
            const int e = k / Q;
            one(k, meta.row[e], queue[k], IMAGE ? meta.w[e] : 1.0f);
        }
    }
    if (lane < E && (uint64_t)(int64_t)meta.row[lane] < (uint64_t)a.n_x)
        red_add_u32(a.cnt + meta.row[lane], meta.n[lane], keep);
}

// One warp's 32 pixels of a tile with a compile-time class count C and LPP
// lanes per pixel, each lane owning QPL = C / (4 LPP) quads (lane q: quads
// q, q + LPP, ...).  The warp runs G = 32 / LPP groups over contiguous pixel
// ranges in lock step, one pixel per group and step.
//  1. Layout, once per tile with lane k looking at pixel k: where entries
//     start and end, each entry's slot (its rank among the tile's entries),
//     row, length and weight -- a few ballots instead of per-step decisions.
//  2. Steps: each lane multiplies (adds) its quads of the group's pixel into
//     the running entry, restarting it where an entry starts, and stores it
//     into the entry's slot where one ends.  No branch depends on a group.
//  3. The warp adds all entries into P (drain).
// queue: the warp's 32-entry array; meta: its entry metadata; release: the
// stage's empty barrier, arrived on once the stage is no longer read (null
// for the ragged tile).
template <int C, int LPP, int RULE, int DT, bool SMEM, bool IMAGE>
__device__ __forceinline__ void warp_tile_q(const ScatterArgs &a, const uint8_t *base, int px0, int lane, int row, float w,
                                            float sc, float4 *queue, EntryMeta &meta, uint64_t *release)
{
    constexpr int ES = Elem<DT>::size;
    constexpr int Q = C / 4;
    constexpr int QPL = Q / LPP;
    constexpr int G = 32 / LPP;
    constexpr int STEPS = (32 + G - 1) / G;  // the longest group range
    constexpr int pstride = C * ES;
    constexpr bool PROD = RULE == SM_RULE_LOGSUM;
    // BF16 / FP8 storage (p = q * scale, one scale per pixel): sum scales in
    // its FMA; max-sum and vote decide on the codes (a positive common scale
    // keeps the order and the ties of a pixel's classes) and scale only the
    // kept maximum; log-sum scales each value before its clamp (measured
    // faster than clamping codes at 2^-30 / scale, which needs per-entry scale
    // products in shared memory).
    constexpr bool SCALED = DT != SM_F32;
    // first and last pixel of every group range
    constexpr uint32_t kFirst = [] {
        uint32_t m = 0;
        for (int g = 0; g < G; ++g) m |= 1u << ((32 * g) / G);
        return m;
    }();
    constexpr uint32_t kLast = [] {
        uint32_t m = 0;
        for (int g = 0; g < G; ++g) m |= 1u << ((32 * (g + 1)) / G - 1);
        return m;
    }();
    const int g = lane / LPP, q = lane - g * LPP;
    const bool active = g < G;
    const int start = active ? (32 * g) / G : 0;
    const int len = active ? (32 * (g + 1)) / G - start : 0;
    const uint8_t *pb = base + (px0 + start) * pstride;
    // register slot m of the lane holds quad qd[m]; odd groups take their
    // quads in the other order, so that the groups of a quarter-warp (whose
    // pixels lie 5-6 pixels apart) spread their 16-byte words over more
    // shared-memory banks: for c = 40 a warp tile's loads take 64 instead of
    // 84 quarter-warp passes (FP32), 44 instead of 64 (BF16), 22 instead of
    // 44 (FP8)
    int qd[QPL];
#pragma unroll
    for (int m = 0; m < QPL; ++m) qd[m] = q + LPP * ((m + g) % QPL);

    // the lane's quads of every step's pixel (a stage holds the whole tile;
    // the ragged tile in global memory is read only where a pixel exists)
    float4 v[STEPS][QPL];
    float sv[STEPS];
#pragma unroll
    for (int u = 0; u < STEPS; ++u) {
        const int k = (start + u) & 31;
        sv[u] = (DT != SM_F32) ? __shfl_sync(kFull, sc, k) : 1.0f;
        const int rk = SMEM ? 0 : __shfl_sync(kFull, row, k);
#pragma unroll
        for (int m = 0; m < QPL; ++m) {
            v[u][m] = make_float4(0.f, 0.f, 0.f, 0.f);
            // FP32 from the stage: only steps inside the group's range are read
            // (an idle lane would take shared-memory bank cycles from its
            // quarter-warp; the values of the other steps are never stored).
            // BF16 / FP8 read every step: there the predicate costs more in
            // branching around the decode than it saves (measured)
            if (SMEM ? (DT != SM_F32 || (active && u < len)) : rk >= 0) {
                v[u][m] = load_quad<DT, SMEM>(pb + u * pstride, 4 * qd[m]);
                if (SCALED && PROD) v[u][m] = scale4(v[u][m], sv[u]);
            }
        }
    }

    // 1. entry layout (lane = pixel)
    const uint32_t le = lane == 31 ? kFull : ((2u << lane) - 1u);  // pixels 0 .. lane
    // (every lane executes every shuffle and ballot: none sits behind a
    // lane-dependent condition)
    const int rprev = __shfl_up_sync(kFull, row, 1);
    const float wprev = IMAGE ? __shfl_up_sync(kFull, w, 1) : w;
    bool brk = ((kFirst >> lane) & 1u) || row != rprev;
    if (IMAGE && w != wprev) brk = true;
    bool first = brk;
    if (PROD) {
        // split runs every kMaxFactors pixels
        const uint32_t B = __ballot_sync(kFull, brk);
        const int pos = lane - (31 - __clz(B & le));
        first = brk || (pos & (kMaxFactors - 1)) == 0;
    }
    const uint32_t S = __ballot_sync(kFull, first);                 // entry (or background run) starts
    const uint32_t R = __ballot_sync(kFull, first && row >= 0);     // entry starts
    const int E = __popc(R);
    const int slot = __popc(R & le) - 1;
    const uint32_t next = lane == 31 ? 0u : (S >> (lane + 1)) & 1u;   // the next pixel starts a run
    const bool last = row >= 0 && (((kLast >> lane) & 1u) || next);
    if (last && slot >= 0) {
        meta.row[slot] = row;
        meta.n[slot] = (uint32_t)(lane - (31 - __clz(S & le)) + 1);
        if (IMAGE) meta.w[slot] = w;
    }
    const int info = (first ? 32 : 0) | (last ? 64 : 0) | (slot & 31);
    __syncwarp();  // every lane's stage reads are done before entries may overwrite them

    // 2. steps
    float4 s[QPL];
#pragma unroll
    for (int m = 0; m < QPL; ++m) s[m] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int u = 0; u < STEPS; ++u) {
        int inf = __shfl_sync(kFull, info, (start + u) & 31);
        if (u >= len) inf = 0;  // past the group's range
        const bool st = inf & 32;
        if (RULE == SM_RULE_SUM) {
#pragma unroll
            for (int m = 0; m < QPL; ++m) {
                if (SCALED) {
                    s[m].x = fmaf(v[u][m].x, sv[u], st ? 0.f : s[m].x);
                    s[m].y = fmaf(v[u][m].y, sv[u], st ? 0.f : s[m].y);
                    s[m].z = fmaf(v[u][m].z, sv[u], st ? 0.f : s[m].z);
                    s[m].w = fmaf(v[u][m].w, sv[u], st ? 0.f : s[m].w);
                } else {
                    s[m].x = st ? v[u][m].x : s[m].x + v[u][m].x;
                    s[m].y = st ? v[u][m].y : s[m].y + v[u][m].y;
                    s[m].z = st ? v[u][m].z : s[m].z + v[u][m].z;
                    s[m].w = st ? v[u][m].w : s[m].w + v[u][m].w;
                }
            }
        } else if (RULE == SM_RULE_LOGSUM) {
#pragma unroll
            for (int m = 0; m < QPL; ++m) {
                const float4 c = make_float4(fmaxf(v[u][m].x, kPMin), fmaxf(v[u][m].y, kPMin),
                                             fmaxf(v[u][m].z, kPMin), fmaxf(v[u][m].w, kPMin));
                s[m].x = st ? c.x : s[m].x * c.x;
                s[m].y = st ? c.y : s[m].y * c.y;
                s[m].z = st ? c.z : s[m].z * c.z;
                s[m].w = st ? c.w : s[m].w * c.w;
            }
        } else {
            // maximum and first arg max of the whole pixel: each lane takes the
            // lowest class among its own maxima (its slots need not be in class
            // order), then the group combines (lowest class on ties); max-sum
            // needs the maximum only
            float mx = -INFINITY;
            int am = 0x7fffffff;
            auto take = [&](float val, int idx) {
                if (val > mx || (RULE == SM_RULE_VOTE && val == mx && idx < am)) {
                    mx = val;
                    am = idx;
                }
            };
#pragma unroll
            for (int m = 0; m < QPL; ++m) {
                const int j = qd[m];
                take(v[u][m].x, 4 * j);
                take(v[u][m].y, 4 * j + 1);
                take(v[u][m].z, 4 * j + 2);
                take(v[u][m].w, 4 * j + 3);
            }
            float gm = mx;
            int ga = am;
#pragma unroll
            for (int t = 0; t < LPP; ++t) {
                const float om = __shfl_sync(kFull, mx, g * LPP + t);
                const int oa = __shfl_sync(kFull, am, g * LPP + t);
                if (om > gm || (om == gm && oa < ga)) {
                    gm = om;
                    ga = oa;
                }
            }
            const float gv = SCALED ? __fmul_rn(gm, sv[u]) : gm;  // the kept maximum, scaled once
#pragma unroll
            for (int m = 0; m < QPL; ++m) {
                const int j = qd[m];
                float4 c;
                if (RULE == SM_RULE_MAXSUM) {
                    c = make_float4(v[u][m].x == gm ? gv : 0.f, v[u][m].y == gm ? gv : 0.f,
                                    v[u][m].z == gm ? gv : 0.f, v[u][m].w == gm ? gv : 0.f);
                } else {
                    c = make_float4(ga == 4 * j ? 1.f : 0.f, ga == 4 * j + 1 ? 1.f : 0.f,
                                    ga == 4 * j + 2 ? 1.f : 0.f, ga == 4 * j + 3 ? 1.f : 0.f);
                }
                s[m].x = st ? c.x : s[m].x + c.x;
                s[m].y = st ? c.y : s[m].y + c.y;
                s[m].z = st ? c.z : s[m].z + c.z;
                s[m].w = st ? c.w : s[m].w + c.w;
            }
        }
        if (inf & 64) {
#pragma unroll
            for (int m = 0; m < QPL; ++m) queue[(inf & 31) * Q + qd[m]] = s[m];
        }
    }
    __syncwarp();

    // 3. drain, then hand the stage back (the entries written into it by
    // plain stores must be ordered before the copy engine's next refill)
    drain<C, RULE, IMAGE, DT == SM_F32>(a, queue, meta, E, lane);
    if (release) {
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) mbar_arrive(release);
    }
}

}  // namespace sdev
}  // namespace lf
