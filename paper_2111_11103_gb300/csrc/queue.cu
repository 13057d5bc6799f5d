// Persistent fusion kernel with a device work queue: the renderer (Sec.
// 3.3.1) and the aggregator's update of the rows of P (Sec. 3.3.2, Eqs. sum /
// mul / maxsum and their weighted forms) of a whole sequence in one launch.
//
// The frames are cut into batches of B frames; batch b renders into z-buffer
// slot b % S.  The queue holds two kinds of work items, taken in order from
// one atomic counter by persistent CTAs (two per SM, each with the scatter's
// shape: a producer warp and 8 consumer warps):
//   raster (b, frame, cluster range): the cluster cull and the raster of up
//     to kCullRound clusters of 32 faces per round into the frame's z-buffer
//     (64-bit red.min keys, as in the stream-ordered raster);
//   scatter (b, tile range): the pipelined scatter of 256-pixel tiles of the
//     batch (TMA bulk copies of predictions and z-buffer keys, entries built
//     in registers, vector reductions into P; the keys are re-armed).
// Order: R(0) .. R(L-1), then R(p), S(p - L) for p = L .. nb-1, then the
// remaining S -- the raster of later batches runs on some CTAs while others
// scatter earlier batches, so raster and scatter overlap on the same SMs,
// and small batches keep the z-buffer slots resident in L2.
// Dependencies, waited for by one thread per CTA before it starts an item:
//   S(b) after every R(b) item (acquire of rdone[b]);
//   R(b) after every S(b - S) item, the last reader of its slot (sdone).
// Each such item lies earlier in the queue (S > L), and an item is taken
// only by a running CTA that never waits for a later item, so the earliest
// unfinished item always progresses: no deadlock for any grid size.  Every
// wait is bounded (kWaitNs); a wait that gives up latches kErrTimeout and
// raises an abort flag that makes every other wait and item of the launch
// give up at once, so a failure drains the launch quickly.
#include <cstdlib>

#include "raster_dev.cuh"
#include "scatter_dev.cuh"

namespace lf {
namespace {

using namespace sdev;

constexpr int kWarps = kThreads / 32;
constexpr int kCullRound = 4 * kThreads;  // clusters tested per raster round
constexpr uint32_t kRasterSmem = 64 + kCullRound * 4;  // camera rows + the round's visible-cluster list

struct QueueArgs {
    // mesh
    const float4 *V;
    const int4 *faces;
    int64_t F, ncl;
    const float4 *bounds;
    const Camera *cams;  // frame 0 of the launch first
    int H, W;
    int64_t npix;
    // predictions of the launch's frames, accumulators
    const uint8_t *probs;
    const float *scale;
    int64_t frame_bytes;  // npix * c * element size
    int c;
    bool scale_bulk;
    int32_t *ids_out;  // optional row maps of the launch's frames
    float *acc;
    uint32_t *cnt;
    int64_t n_x;
    int32_t *err;
    // z-buffer slots (S of slot_stride keys each; all keys empty on entry)
    unsigned long long *keys;
    int64_t slot_stride;
    int slots;
    // plan
    int nb, B;             // batches, frames per batch
    int rpf, rchunk;       // raster items per frame, clusters per raster item
    uint32_t nR, nS;       // items per batch
    int schunk;            // tiles per scatter item
    int lookahead;         // L
    int64_t tiles_full;    // full 256-pixel tiles per batch
    bool ragged;           // a batch ends with a partial tile
    // queue state (zeroed before the launch): head, rdone[nb], sdone[nb], abort
    uint32_t *head, *rdone, *sdone;
    int32_t *abort;
    uint64_t wait_ns;
    int skip_it;           // test hook: the producer leaves this ring step unfilled (-1: never)
};

// Item i of the queue -> (kind 0 = raster / 1 = scatter, batch, index within
// the batch's items of that kind); closed form of the order described above.
__device__ __forceinline__ void decode(const QueueArgs &q, uint32_t i, int &kind, int &b, uint32_t &sub)
{
    const uint32_t L = (uint32_t)q.lookahead, nb = (uint32_t)q.nb, nR = q.nR, nS = q.nS;
    const uint32_t A = L < nb ? L : nb;
    if (i < A * nR) {
        kind = 0;
        b = (int)(i / nR);
        sub = i % nR;
        return;
    }
    i -= A * nR;
    const uint32_t M = nb > L ? nb - L : 0u;
    if (i < M * (nR + nS)) {
        const uint32_t p = L + i / (nR + nS), r = i % (nR + nS);
        if (r < nR) {
            kind = 0;
            b = (int)p;
            sub = r;
        } else {
            kind = 1;
            b = (int)(p - L);
            sub = r - nR;
        }
        return;
    }
    i -= M * (nR + nS);
    kind = 1;
    b = (int)(M + i / nS);
    sub = i % nS;
}

__device__ __forceinline__ bool aborted(const QueueArgs &q) { return *(volatile const int32_t *)q.abort != 0; }

__device__ __forceinline__ void give_up(const QueueArgs &q)
{
    atomicCAS(q.err, 0, (int32_t)kErrTimeout);
    atomicExch(q.abort, 1);
}

// Waits (bounded, abortable) until *ctr >= need; acquire semantics.
__device__ __forceinline__ bool wait_count(const QueueArgs &q, const uint32_t *ctr, uint32_t need)
{
    if (ld_acquire_gpu(ctr) >= need) return true;
    const uint64_t t0 = global_ns();
    for (;;) {
        if (ld_acquire_gpu(ctr) >= need) return true;
        if (aborted(q) || global_ns() - t0 > q.wait_ns) return false;
        __nanosleep(200);
    }
}

// mbarrier phase wait, bounded and abortable.
__device__ __forceinline__ bool mbar_wait_q(const QueueArgs &q, uint64_t *bar, uint32_t parity)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    while (!mbar_try_wait(bar, parity)) {
        if (aborted(q) || global_ns() - t0 > q.wait_ns) return false;
    }
    return true;
}

// Arguments of the stream-ordered scatter for batch b of the launch.
__device__ __forceinline__ ScatterArgs batch_args(const QueueArgs &q, int b)
{
    const int64_t f0 = (int64_t)b * q.B;
    ScatterArgs a;
    a.probs = q.probs + f0 * q.frame_bytes;
    a.scale = q.scale ? q.scale + f0 * q.npix : nullptr;
    a.keys = q.keys + (int64_t)(b % q.slots) * q.slot_stride;
    a.ids_in = nullptr;
    a.ids_out = q.ids_out ? q.ids_out + f0 * q.npix : nullptr;
    a.total_px = (int64_t)q.B * q.npix;
    a.npix = q.npix;
    a.c = q.c;
    a.fcnt = nullptr;
    a.alpha = 1.0f;
    a.wpix = nullptr;
    a.n_x = q.n_x;
    a.acc = q.acc;
    a.cnt = q.cnt;
    a.err = q.err;
    a.scale_bulk = q.scale_bulk;
    a.wait_ns = q.wait_ns;
    a.skip_it = q.skip_it;
    return a;
}

template <int RULE, int DT, int C>
__global__ void __launch_bounds__(kThreads, 2) k_fuse_queue(QueueArgs q, int stages)
{
    extern __shared__ __align__(128) uint8_t smem[];
    // [0, 64): ring barriers (stages <= 4); [64, 128): item broadcast and the
    // raster round's list length; then the entry arrays, the raster area and
    // the ring stages
    uint64_t *full = reinterpret_cast<uint64_t *>(smem);
    uint64_t *empty = full + stages;
    volatile uint32_t *bcast = reinterpret_cast<volatile uint32_t *>(smem + 64);
    uint32_t *s_n = reinterpret_cast<uint32_t *>(smem + 72);
    float *sA = reinterpret_cast<float *>(smem + 128 + EntryLayout<C, DT>::bytes);
    int32_t *s_list = reinterpret_cast<int32_t *>(smem + 128 + EntryLayout<C, DT>::bytes + 64);
    uint8_t *stage0 = smem + 128 + EntryLayout<C, DT>::bytes + ((kRasterSmem + 127u) & ~127u);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t total = (uint32_t)q.nb * (q.nR + q.nS);

    ScatterArgs a0 = batch_args(q, 0);
    const StageLayout L = stage_layout<DT>(a0);
    if (threadIdx.x == 0) {
        for (int s = 0; s < stages; ++s) {
            mbar_init(full + s, 1);
            mbar_init(empty + s, kConsumerWarps);
        }
        fence_mbar_init();
    }
    __syncthreads();

    const int px0 = (warp - 1) * 32;
    EntryMeta &meta = reinterpret_cast<EntryMeta *>(smem + 128)[warp > 0 ? warp - 1 : 0];
    float4 *own_queue = reinterpret_cast<float4 *>(smem + 128 + EntryLayout<C, DT>::kMetaBytes) +
                        (warp > 0 ? warp - 1 : 0) * 8 * C;
    int it = 0;  // ring step: the producer lane and every consumer thread count the same tiles

    for (;;) {
        if (threadIdx.x == 0) {
            const uint32_t i = atomicAdd(q.head, 1u);
            uint32_t ok = 0;
            if (i < total) {
                int kind, b;
                uint32_t sub;
                decode(q, i, kind, b, sub);
                if (kind == 1) ok = wait_count(q, q.rdone + b, q.nR);
                else if (b >= q.slots) ok = wait_count(q, q.sdone + (b - q.slots), q.nS);
                else ok = !aborted(q);
                if (!ok && !aborted(q)) give_up(q);
                if (ok && kind == 1) fence_proxy_async_global();  // keys rendered by other CTAs -> bulk copies
            }
            bcast[0] = i;
            bcast[1] = ok;
        }
        __syncthreads();
        const uint32_t i = bcast[0];
        const bool ok = bcast[1] != 0;
        if (i >= total) break;
        int kind, b;
        uint32_t sub;
        decode(q, i, kind, b, sub);

        if (ok && kind == 0) {
            // ---- raster item: one frame, clusters [c0, c1) ----
            const int fb = (int)(sub / (uint32_t)q.rpf), k = (int)(sub % (uint32_t)q.rpf);
            const int64_t f = (int64_t)b * q.B + fb;
            unsigned long long *fkeys = q.keys + (int64_t)(b % q.slots) * q.slot_stride + (int64_t)fb * q.npix;
            if (threadIdx.x < 12) sA[threadIdx.x] = q.cams[f].a[threadIdx.x];
            const int64_t c0 = (int64_t)k * q.rchunk;
            const int64_t c1 = c0 + q.rchunk < q.ncl ? c0 + q.rchunk : q.ncl;
            for (int64_t base = c0; base < c1; base += kCullRound) {
                if (threadIdx.x == 0) *s_n = 0;
                __syncthreads();  // camera rows and the cleared count visible
#pragma unroll
                for (int r = 0; r < kCullRound / kThreads; ++r) {
                    const int64_t cl = base + r * kThreads + threadIdx.x;
                    const bool keep = cl < c1 && cluster_may_be_visible(q.bounds, cl, sA, q.H, q.W);
                    const unsigned mask = __ballot_sync(kFull, keep);
                    if (mask) {
                        uint32_t at = 0;
                        if (lane == __ffs(mask) - 1) at = atomicAdd(s_n, (uint32_t)__popc(mask));
                        at = __shfl_sync(kFull, at, __ffs(mask) - 1);
                        if (keep) s_list[at + __popc(mask & ((1u << lane) - 1u))] = (int32_t)cl;
                    }
                }
                __syncthreads();
                const uint32_t n = *s_n;
                for (uint32_t j = warp; j < n; j += kWarps)
                    raster_face(sA, q.V, q.faces, q.F, (int64_t)s_list[j] * kClusterFaces + lane, q.H, q.W, fkeys);
                __syncthreads();  // the list is reused by the next round
            }
        } else if (ok) {
            // ---- scatter item: tiles [t0, t1) of batch b ----
            const ScatterArgs a = batch_args(q, b);
            const int64_t t0 = (int64_t)sub * q.schunk;
            const int64_t tiles_b = q.tiles_full + (q.ragged ? 1 : 0);
            const int64_t t1 = t0 + q.schunk < tiles_b ? t0 + q.schunk : tiles_b;
            const int64_t tf1 = t1 < q.tiles_full ? t1 : q.tiles_full;
            if (warp == 0) {
                if (lane == 0) {
                    const uint64_t pol = l2_evict_first();
                    const uint32_t tx = L.probs_bytes + L.meta_bytes + L.scale_bytes;
                    bool failed = false;
                    for (int64_t t = t0; t < tf1; ++t, ++it) {
                        const int s = it % stages;
                        const uint32_t ph = (uint32_t)(it / stages) & 1u;
                        if (it >= stages && !mbar_wait_q(q, empty + s, ph ^ 1u)) {
                            if (!aborted(q)) give_up(q);
                            failed = true;
                            break;
                        }
                        if (it == q.skip_it) continue;  // test hook: this stage is never filled
                        uint8_t *st = stage0 + (size_t)s * L.stride;
                        mbar_arrive_expect_tx(full + s, tx);
                        bulk_g2s(st, a.probs + (size_t)t * L.probs_bytes, L.probs_bytes, full + s, pol);
                        bulk_g2s(st + L.probs_bytes, a.keys + t * kTile, L.meta_bytes, full + s, pol);
                        if (L.scale_bytes)
                            bulk_g2s(st + L.probs_bytes + L.meta_bytes, a.scale + t * kTile, L.scale_bytes, full + s,
                                     pol);
                    }
                    if (failed || aborted(q)) {
                        // every issued copy lands before the CTA moves on
                        for (int j = it - stages; j < it; ++j) {
                            if (j < 0 || j == q.skip_it) continue;
                            if (!mbar_wait(full + (j % stages), (uint32_t)(j / stages) & 1u, q.wait_ns))
                                atomicCAS(q.err, 0, (int32_t)kErrTimeout);
                        }
                    }
                }
            } else {
                bool failed = false;
                for (int64_t t = t0; t < tf1; ++t, ++it) {
                    const int s = it % stages;
                    const uint32_t ph = (uint32_t)(it / stages) & 1u;
                    const uint8_t *st = stage0 + (size_t)s * L.stride;
                    if (!mbar_wait_q(q, full + s, ph)) {
                        if (!aborted(q)) give_up(q);
                        failed = true;
                        break;
                    }
                    int row;
                    float w, sc;
                    pixel_info<DT, false>(
                        a, t * kTile + px0 + lane, px0 + lane, st + L.probs_bytes,
                        L.scale_bytes ? reinterpret_cast<const float *>(st + L.probs_bytes + L.meta_bytes) : nullptr,
                        row, w, sc);
                    float4 *queue = EntryLayout<C, DT>::kInStage
                                        ? reinterpret_cast<float4 *>(const_cast<uint8_t *>(st) + px0 * C * 4)
                                        : own_queue;
                    warp_tile_q<C, 5, RULE, DT, true, false>(a, st, px0, lane, row, w, sc, queue, meta, empty + s);
                }
                if (!failed && t1 > q.tiles_full) {
                    // the batch's partial last tile, from global memory; every
                    // copy of this item has landed and been consumed, so the
                    // warp's slice of stage 0 is free for its entries
                    int row;
                    float w, sc;
                    pixel_info<DT, false>(a, q.tiles_full * kTile + px0 + lane, px0 + lane, nullptr, nullptr, row, w,
                                          sc);
                    float4 *queue = EntryLayout<C, DT>::kInStage ? reinterpret_cast<float4 *>(stage0 + px0 * C * 4)
                                                                 : own_queue;
                    warp_tile_q<C, 5, RULE, DT, false, false>(a, a.probs + (size_t)q.tiles_full * L.probs_bytes, px0,
                                                              lane, row, w, sc, queue, meta, nullptr);
                }
            }
        }
        __syncthreads();  // the item is done by every thread of the CTA
        if (threadIdx.x == 0 && ok && !aborted(q)) {
            __threadfence();  // release: its z-buffer writes / re-arms before the count
            atomicAdd(kind == 0 ? q.rdone + b : q.sdone + b, 1u);
        }
    }
}

struct DevInfoQ {
    int sms;
    uint32_t cta_smem;
};

DevInfoQ dev_info_q()
{
    static std::atomic<uint64_t> known{0};
    static DevInfoQ info[64];
    const int dev = current_device() & 63;
    if (!(known.load() & (1ull << dev))) {
        int sms = 0, per_sm = 0, reserved = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
        const int cta = per_sm / 2 - reserved;
        info[dev] = DevInfoQ{sms > 0 ? sms : 1, cta > (96 << 10) ? (uint32_t)cta : (96u << 10)};
        known.fetch_or(1ull << dev);
    }
    return info[dev];
}

template <int RULE, int DT, int C>
void launch_q(const QueueArgs &q, cudaStream_t s)
{
    static PerDeviceOnce configured;
    const DevInfoQ di = dev_info_q();
    ScatterArgs a0{};
    a0.c = q.c;
    a0.keys = q.keys;
    a0.scale_bulk = q.scale_bulk;
    const StageLayout L = stage_layout<DT>(a0);
    const uint32_t fixed = 128u + EntryLayout<C, DT>::bytes + ((kRasterSmem + 127u) & ~127u);
    int stages = (int)((di.cta_smem - fixed) / L.stride);
    stages = stages < 1 ? 1 : (stages > 4 ? 4 : stages);
    const size_t smem = fixed + (size_t)stages * L.stride;
    if (configured.first(current_device())) {
        cudaFuncSetAttribute(k_fuse_queue<RULE, DT, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 << 10);
        cudaFuncSetAttribute(k_fuse_queue<RULE, DT, C>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
    }
    const int64_t items = (int64_t)q.nb * (q.nR + q.nS);
    int64_t grid = 2LL * di.sms;
    if (grid > items) grid = items;
    if (grid < 1) grid = 1;
    k_fuse_queue<RULE, DT, C><<<(unsigned)grid, kThreads, smem, s>>>(q, stages);
}

template <int RULE, int DT>
void launch_qc(const QueueArgs &q, cudaStream_t s)
{
    if (q.c == 40) launch_q<RULE, DT, 40>(q, s);
    else launch_q<RULE, DT, 20>(q, s);
}

template <int RULE>
void launch_qd(sm_dtype dt, const QueueArgs &q, cudaStream_t s)
{
    if (dt == SM_F32) launch_qc<RULE, SM_F32>(q, s);
    else if (dt == SM_BF16) launch_qc<RULE, SM_BF16>(q, s);
    else launch_qc<RULE, SM_FP8_E4M3>(q, s);
}

}  // namespace

bool fuse_queue_supported(int c) { return c == 40 || c == 20; }

int fuse_queue_raster_round() { return kCullRound; }

uint32_t fuse_queue_counter_words(int nb) { return 2u * (uint32_t)nb + 2u; }

void launch_fuse_queue(const FuseQueueLaunch &l, cudaStream_t s)
{
    if (l.nb <= 0 || l.npix <= 0) return;
    QueueArgs q{};
    q.V = l.V;
    q.faces = l.faces;
    q.F = l.F;
    q.ncl = (l.F + kClusterFaces - 1) / kClusterFaces;
    q.bounds = l.bounds;
    q.cams = l.cams;
    q.H = l.H;
    q.W = l.W;
    q.npix = l.npix;
    q.probs = static_cast<const uint8_t *>(l.probs);
    q.scale = l.scale;
    q.c = l.c;
    q.frame_bytes = l.npix * l.c * (l.dtype == SM_F32 ? 4 : (l.dtype == SM_BF16 ? 2 : 1));
    q.scale_bulk = l.scale != nullptr && ((uintptr_t)l.scale & 15) == 0;
    q.ids_out = l.ids_out;
    q.acc = l.acc;
    q.cnt = l.cnt;
    q.n_x = l.n_x;
    q.err = l.err;
    q.keys = l.keys;
    q.slot_stride = l.slot_stride;
    q.slots = l.lookahead + 2;
    q.nb = l.nb;
    q.B = l.B;
    q.rchunk = l.raster_rounds * kCullRound;
    q.rpf = (int)((q.ncl + q.rchunk - 1) / q.rchunk);
    q.nR = (uint32_t)(q.rpf * l.B);
    q.tiles_full = (int64_t)l.B * l.npix / kTile;
    q.ragged = q.tiles_full * kTile < (int64_t)l.B * l.npix;
    q.schunk = l.scatter_tiles;
    q.nS = (uint32_t)((q.tiles_full + (q.ragged ? 1 : 0) + q.schunk - 1) / q.schunk);
    q.lookahead = l.lookahead;
    q.head = l.counters;
    q.rdone = l.counters + 1;
    q.sdone = l.counters + 1 + l.nb;
    q.abort = reinterpret_cast<int32_t *>(l.counters + 1 + 2 * l.nb);
    q.wait_ns = kWaitNs;
    q.skip_it = -1;
    // Test hook, as in the stream-ordered scatter (LABELFUSE_TEST_SKIP_TILE=k):
    // every CTA's producer leaves its k-th ring step unfilled and waits give
    // up after 5 ms; the launch then drains through the abort flag.
    if (const char *env = getenv("LABELFUSE_TEST_SKIP_TILE")) {
        q.skip_it = atoi(env);
        q.wait_ns = 5000000ull;
    }
    cudaMemsetAsync(l.counters, 0, fuse_queue_counter_words(l.nb) * sizeof(uint32_t), s);
    switch (l.rule) {
    case SM_RULE_SUM: launch_qd<SM_RULE_SUM>(l.dtype, q, s); break;
    case SM_RULE_LOGSUM: launch_qd<SM_RULE_LOGSUM>(l.dtype, q, s); break;
    case SM_RULE_MAXSUM: launch_qd<SM_RULE_MAXSUM>(l.dtype, q, s); break;
    default: launch_qd<SM_RULE_VOTE>(l.dtype, q, s); break;
    }
}

}  // namespace lf
