// Persistent fusion kernel with a device work queue: the renderer (Sec.
// 3.3.1) and the aggregator's update of the rows of P (Sec. 3.3.2, Eqs. sum /
// mul / maxsum and their weighted forms) of whole sequences in one launch --
// one scene, or up to kMaxScenes independent scenes (each its own mesh,
// accumulators, frames and image size), so no launch boundary separates
// batches or scenes.
//
// Each scene's frames are cut into batches of its B frames; batch b of a
// scene renders into that scene's z-buffer slot b % S.  The launch treats the
// batches of all its scenes as one sequence g = 0 .. G-1 (scene after scene).
// The queue holds two kinds of work items, taken in order from one atomic
// counter by persistent CTAs (two per SM, each with the scatter's shape: a
// producer warp and 8 consumer warps):
//   raster R(g): (frame, cluster range) -- the cluster cull and the raster of
//     up to kCullRound clusters of 32 faces per round into the frame's
//     z-buffer (64-bit red.min keys, as in the stream-ordered raster);
//   scatter S(g): a range of 256-pixel tiles of the batch -- the pipelined
//     scatter (TMA bulk copies of predictions and z-buffer keys, entries built
//     in registers, vector reductions into P; the keys are re-armed).
// Order, in phases p = 0 .. G+L-1: phase p holds the items of R(p) (p < G)
// spread evenly among those of S(p - L) (p >= L; a raster item after every
// nS / nR scatter items, Bresenham spacing).  So at any moment about the
// raster's share of the CTAs renders later batches (or the next scene) while
// the others scatter earlier ones, and small batches keep the z-buffer slots
// resident in L2.
// Dependencies, waited for by one thread per CTA before it starts an item:
//   S(g) after every R(g) item (acquire of rdone[g]);
//   R(g) after every S(g - S) item when g - S is a batch of the same scene,
//   the last reader of its slot (sdone).
// Each such item lies in an earlier phase (L >= 1, S > L), and an item is
// taken only by a running CTA that never waits for a later item, so the
// earliest unfinished item always progresses: no deadlock for any grid size.
// Every wait is bounded (kWaitNs); a wait that gives up latches kErrTimeout
// and raises an abort flag that makes every other wait and item of the
// launch give up at once, so a failure drains the launch quickly.
#include <cstdlib>

#include "raster_dev.cuh"
#include "scatter_dev.cuh"

namespace lf {
namespace {

using namespace sdev;

constexpr int kWarps = kThreads / 32;
constexpr int kCullRound = 4 * kThreads;  // clusters tested per raster round
constexpr uint32_t kRasterSmem = 64 + kCullRound * 4;  // camera rows + the round's visible-cluster list

// One scene of a launch (per-scene plan and buffers).
struct QueueScene {
    // mesh
    const float4 *V;
    const int4 *faces;
    int64_t F, ncl;
    const float4 *bounds;
    const Camera *cams;  // the scene's first frame of the launch first
    int H, W;
    int64_t npix;
    // predictions of the launch's frames, accumulators
    const uint8_t *probs;
    const float *scale;
    int64_t frame_bytes;  // npix * c * element size
    int32_t *ids_out;  // optional row maps of the launch's frames
    float *acc;
    uint32_t *cnt;
    int64_t n_x;
    int32_t *err;
    // z-buffer slots (slots of slot_stride keys each; all keys empty on entry)
    unsigned long long *keys;
    int64_t slot_stride;
    // plan
    int slots;
    int B;                 // frames per batch
    int rpf, rchunk;       // raster items per frame, clusters per raster item
    uint32_t nR, nS;       // items per batch
    int schunk;            // tiles per scatter item
    int64_t tiles_full;    // full 256-pixel tiles per batch
    int ragged;            // a batch ends with a partial tile
};

constexpr int kMaxScenes = 12;
constexpr int kMaxBatches = 128;     // batches (all scenes) per launch
constexpr int kMaxLookahead = 4;

// Everything a launch needs, passed by value (read in place: __grid_constant__).
struct QueueArgs {
    QueueScene sc[kMaxScenes];
    int batch0[kMaxScenes + 1];      // first batch g of every scene; batch0[nscenes] = G
    uint32_t phase0[kMaxBatches + kMaxLookahead + 1];  // first item of every phase; phase0[G + L] = total
    int nscenes, G, L;
    int c;
    bool scale_bulk;                 // per-pixel scales copied with the tiles (all scenes 16-byte aligned)
    uint32_t *head;                  // queue head (zeroed before the launch)
    int32_t *abort;                  // raised by a wait that gave up
    uint32_t *rdone, *sdone;         // completion counts per batch g (zeroed before the launch)
    uint64_t wait_ns;
    int skip_it;                     // test hook: the producer leaves this ring step unfilled (-1: never)
};
static_assert(sizeof(QueueArgs) <= 4000, "kernel parameters stay within 4 KB");

// Scene of batch g and its index b within the scene.
__device__ __forceinline__ int scene_of_batch(const QueueArgs &q, int g, int &b)
{
    int s = 0;
    while (s + 1 < q.nscenes && g >= q.batch0[s + 1]) ++s;
    b = g - q.batch0[s];
    return s;
}

// Item i of the launch -> (kind 0 = raster / 1 = scatter, batch g, index
// within the batch's items of that kind); the phase order described above.
__device__ __forceinline__ void decode(const QueueArgs &q, uint32_t i, int &kind, int &g, uint32_t &sub)
{
    // the phase holding item i: the last p with phase0[p] <= i
    int lo = 0, hi = q.G + q.L - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (q.phase0[mid] <= i) lo = mid;
        else hi = mid - 1;
    }
    const int p = lo;
    const uint32_t r = i - q.phase0[p];
    int b;
    const uint32_t nR = p < q.G ? q.sc[scene_of_batch(q, p, b)].nR : 0u;
    const uint32_t nS = p >= q.L ? q.sc[scene_of_batch(q, p - q.L, b)].nS : 0u;
    const uint32_t T = nR + nS;
    // raster items among the first r positions of the phase: floor(r nR / T)
    const uint32_t kr = (uint32_t)(((uint64_t)r * nR) / T);
    const uint32_t kr1 = (uint32_t)(((uint64_t)(r + 1) * nR) / T);
    if (kr1 > kr) {
        kind = 0;
        g = p;
        sub = kr;
    } else {
        kind = 1;
        g = p - q.L;
        sub = r - kr;
    }
}

__device__ __forceinline__ bool aborted(const QueueArgs &q) { return *(volatile const int32_t *)q.abort != 0; }

__device__ __forceinline__ void give_up(const QueueArgs &q, int32_t *err)
{
    atomicCAS(err, 0, (int32_t)kErrTimeout);
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

// Arguments of the stream-ordered scatter for batch b of scene q.
__device__ __forceinline__ ScatterArgs batch_args(const QueueArgs &la, const QueueScene &q, int b)
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
    a.c = la.c;
    a.fcnt = nullptr;
    a.alpha = 1.0f;
    a.wpix = nullptr;
    a.n_x = q.n_x;
    a.acc = q.acc;
    a.cnt = q.cnt;
    a.err = q.err;
    a.scale_bulk = la.scale_bulk;
    a.wait_ns = la.wait_ns;
    a.skip_it = la.skip_it;
    return a;
}

template <int RULE, int DT, int C>
__global__ void __launch_bounds__(kThreads, 2) k_fuse_queue(const __grid_constant__ QueueArgs q, int stages)
{
    extern __shared__ __align__(128) uint8_t smem[];
    // [0, 64): ring barriers (stages <= 4); [64, 128): item broadcast and the
    // raster round's list length; then the entry arrays, the raster area and
    // the ring stages
    uint64_t *full = reinterpret_cast<uint64_t *>(smem);
    uint64_t *empty = full + stages;
    volatile uint32_t *bcast = reinterpret_cast<volatile uint32_t *>(smem + 64);  // item, ok, kind, g, sub
    uint32_t *s_n = reinterpret_cast<uint32_t *>(smem + 96);
    float *sA = reinterpret_cast<float *>(smem + 128 + EntryLayout<C, DT>::bytes);
    int32_t *s_list = reinterpret_cast<int32_t *>(smem + 128 + EntryLayout<C, DT>::bytes + 64);
    uint8_t *stage0 = smem + 128 + EntryLayout<C, DT>::bytes + ((kRasterSmem + 127u) & ~127u);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t total = q.phase0[q.G + q.L];

    ScatterArgs a0 = batch_args(q, q.sc[0], 0);  // the stage layout is the same for every scene of the launch
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
            int kind = 0, g = 0;
            uint32_t sub = 0;
            if (i < total) {
                decode(q, i, kind, g, sub);
                int b;
                const QueueScene &sq = q.sc[scene_of_batch(q, g, b)];
                if (kind == 1) ok = wait_count(q, q.rdone + g, sq.nR);
                else if (b >= sq.slots) ok = wait_count(q, q.sdone + (g - sq.slots), sq.nS);
                else ok = !aborted(q);
                if (!ok && !aborted(q)) give_up(q, sq.err);
                if (ok && kind == 1) fence_proxy_async_global();  // keys rendered by other CTAs -> bulk copies
            }
            bcast[0] = i;
            bcast[1] = ok;
            bcast[2] = (uint32_t)kind;
            bcast[3] = (uint32_t)g;
            bcast[4] = sub;
        }
        __syncthreads();
        const uint32_t i = bcast[0];
        const bool ok = bcast[1] != 0;
        if (i >= total) break;
        const int kind = (int)bcast[2], g = (int)bcast[3];
        const uint32_t sub = bcast[4];
        int b;
        const QueueScene &sq = q.sc[scene_of_batch(q, g, b)];

        if (ok && kind == 0) {
            // ---- raster item: one frame, clusters [c0, c1) ----
            const int fb = (int)(sub / (uint32_t)sq.rpf), k = (int)(sub % (uint32_t)sq.rpf);
            const int64_t f = (int64_t)b * sq.B + fb;
            unsigned long long *fkeys = sq.keys + (int64_t)(b % sq.slots) * sq.slot_stride + (int64_t)fb * sq.npix;
            if (threadIdx.x < 12) sA[threadIdx.x] = sq.cams[f].a[threadIdx.x];
            const int64_t c0 = (int64_t)k * sq.rchunk;
            const int64_t c1 = c0 + sq.rchunk < sq.ncl ? c0 + sq.rchunk : sq.ncl;
            for (int64_t base = c0; base < c1; base += kCullRound) {
                if (threadIdx.x == 0) *s_n = 0;
                __syncthreads();  // camera rows and the cleared count visible
#pragma unroll
                for (int r = 0; r < kCullRound / kThreads; ++r) {
                    const int64_t cl = base + r * kThreads + threadIdx.x;
                    const bool keep = cl < c1 && cluster_may_be_visible(sq.bounds, cl, sA, sq.H, sq.W);
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
                    raster_face(sA, sq.V, sq.faces, sq.F, (int64_t)s_list[j] * kClusterFaces + lane, sq.H, sq.W, fkeys);
                __syncthreads();  // the list is reused by the next round
            }
        } else if (ok) {
            // ---- scatter item: tiles [t0, t1) of batch b ----
            const ScatterArgs a = batch_args(q, sq, b);
            const int64_t t0 = (int64_t)sub * sq.schunk;
            const int64_t tiles_b = sq.tiles_full + (sq.ragged ? 1 : 0);
            const int64_t t1 = t0 + sq.schunk < tiles_b ? t0 + sq.schunk : tiles_b;
            const int64_t tf1 = t1 < sq.tiles_full ? t1 : sq.tiles_full;
            if (warp == 0) {
                if (lane == 0) {
                    const uint64_t pol = l2_evict_first();
                    const uint32_t tx = L.probs_bytes + L.meta_bytes + L.scale_bytes;
                    bool failed = false;
                    for (int64_t t = t0; t < tf1; ++t, ++it) {
                        const int s = it % stages;
                        const uint32_t ph = (uint32_t)(it / stages) & 1u;
                        if (it >= stages && !mbar_wait_q(q, empty + s, ph ^ 1u)) {
                            if (!aborted(q)) give_up(q, sq.err);
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
                                atomicCAS(sq.err, 0, (int32_t)kErrTimeout);
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
                        if (!aborted(q)) give_up(q, sq.err);
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
                if (!failed && t1 > sq.tiles_full) {
                    // the batch's partial last tile, from global memory; every
                    // copy of this item has landed and been consumed, so the
                    // warp's slice of stage 0 is free for its entries
                    int row;
                    float w, sc;
                    pixel_info<DT, false>(a, sq.tiles_full * kTile + px0 + lane, px0 + lane, nullptr, nullptr, row, w,
                                          sc);
                    float4 *queue = EntryLayout<C, DT>::kInStage ? reinterpret_cast<float4 *>(stage0 + px0 * C * 4)
                                                                 : own_queue;
                    warp_tile_q<C, 5, RULE, DT, false, false>(a, a.probs + (size_t)sq.tiles_full * L.probs_bytes, px0,
                                                              lane, row, w, sc, queue, meta, nullptr);
                }
            }
        }
        __syncthreads();  // the item is done by every thread of the CTA
        if (threadIdx.x == 0 && ok && !aborted(q)) {
            __threadfence();  // release: its z-buffer writes / re-arms before the count
            atomicAdd(kind == 0 ? q.rdone + g : q.sdone + g, 1u);
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
    a0.keys = q.sc[0].keys;
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
    const int64_t items = q.phase0[q.G + q.L];
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

int fuse_queue_max_scenes() { return kMaxScenes; }

int fuse_queue_max_batches() { return kMaxBatches; }

uint32_t fuse_queue_counter_words(int G) { return 2u + 2u * (uint32_t)G; }

bool launch_fuse_queue(const FuseQueueScene *scenes, int n, sm_dtype dtype, int c, sm_rule rule, int lookahead,
                       uint32_t *counters, cudaStream_t s)
{
    if (n <= 0 || n > kMaxScenes || lookahead < 1 || lookahead > kMaxLookahead) return false;
    QueueArgs q{};
    q.c = c;
    q.scale_bulk = true;
    q.L = lookahead;
    const int64_t esz = dtype == SM_F32 ? 4 : (dtype == SM_BF16 ? 2 : 1);
    int used = 0, G = 0;
    for (int k = 0; k < n; ++k) {
        const FuseQueueScene &l = scenes[k];
        if (l.nb <= 0 || l.npix <= 0) continue;
        if (G + l.nb > kMaxBatches) return false;  // the caller splits larger launches
        QueueScene &sc = q.sc[used];
        sc.V = l.V;
        sc.faces = l.faces;
        sc.F = l.F;
        sc.ncl = (l.F + kClusterFaces - 1) / kClusterFaces;
        sc.bounds = l.bounds;
        sc.cams = l.cams;
        sc.H = l.H;
        sc.W = l.W;
        sc.npix = l.npix;
        sc.probs = static_cast<const uint8_t *>(l.probs);
        sc.scale = l.scale;
        sc.frame_bytes = l.npix * c * esz;
        if (l.scale == nullptr || ((uintptr_t)l.scale & 15) != 0) q.scale_bulk = false;
        sc.ids_out = l.ids_out;
        sc.acc = l.acc;
        sc.cnt = l.cnt;
        sc.n_x = l.n_x;
        sc.err = l.err;
        sc.keys = l.keys;
        sc.slot_stride = l.slot_stride;
        sc.slots = l.slots;
        sc.B = l.B;
        sc.rchunk = l.raster_rounds * kCullRound;
        sc.rpf = (int)((sc.ncl + sc.rchunk - 1) / sc.rchunk);
        sc.nR = (uint32_t)(sc.rpf * l.B);
        sc.tiles_full = (int64_t)l.B * l.npix / kTile;
        sc.ragged = sc.tiles_full * kTile < (int64_t)l.B * l.npix;
        sc.schunk = l.scatter_tiles;
        sc.nS = (uint32_t)((sc.tiles_full + (sc.ragged ? 1 : 0) + sc.schunk - 1) / sc.schunk);
        if (sc.slots <= q.L) return false;  // the order's deadlock freedom needs S > L
        q.batch0[used] = G;
        G += l.nb;
        ++used;
    }
    if (used == 0) return true;
    q.nscenes = used;
    q.batch0[used] = G;
    q.G = G;
    // phase p: the raster items of batch p and the scatter items of batch p - L
    uint32_t total = 0;
    for (int p = 0; p < G + q.L; ++p) {
        q.phase0[p] = total;
        int s = 0;
        if (p < G) {
            while (s + 1 < used && p >= q.batch0[s + 1]) ++s;
            total += q.sc[s].nR;
        }
        if (p >= q.L) {
            s = 0;
            while (s + 1 < used && p - q.L >= q.batch0[s + 1]) ++s;
            total += q.sc[s].nS;
        }
    }
    q.phase0[G + q.L] = total;
    if (dtype == SM_F32) q.scale_bulk = false;
    q.head = counters;
    q.abort = reinterpret_cast<int32_t *>(counters + 1);
    q.rdone = counters + 2;
    q.sdone = counters + 2 + G;
    q.wait_ns = kWaitNs;
    q.skip_it = -1;
    // Test hook, as in the stream-ordered scatter (LABELFUSE_TEST_SKIP_TILE=k):
    // every CTA's producer leaves its k-th ring step unfilled and waits give
    // up after 5 ms; the launch then drains through the abort flag.
    if (const char *env = getenv("LABELFUSE_TEST_SKIP_TILE")) {
        q.skip_it = atoi(env);
        q.wait_ns = 5000000ull;
    }
    cudaMemsetAsync(counters, 0, fuse_queue_counter_words(G) * sizeof(uint32_t), s);
    switch (rule) {
    case SM_RULE_SUM: launch_qd<SM_RULE_SUM>(dtype, q, s); break;
    case SM_RULE_LOGSUM: launch_qd<SM_RULE_LOGSUM>(dtype, q, s); break;
    case SM_RULE_MAXSUM: launch_qd<SM_RULE_MAXSUM>(dtype, q, s); break;
    default: launch_qd<SM_RULE_VOTE>(dtype, q, s); break;
    }
    return true;
}

}  // namespace lf
