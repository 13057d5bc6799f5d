// C ABI of the label-fusion library: argument validation, library-owned
// buffers, batching of frames and the launch sequence of the hot path
// (camera set-up -> raster -> resolve -> [row histogram] -> scatter), plus
// normalisation, render-back, state import/export and kernel timing.
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <unordered_map>
#include <vector>

#include <cuda.h>  // driver types of the virtual-memory calls (entry points fetched at run time)
#include <nvtx3/nvToolsExt.h>  // header-only; inert unless a profiler attaches

#include "lf_internal.cuh"

namespace {

thread_local char g_last_error[512] = "";

sm_status fail(sm_status st, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof g_last_error, fmt, ap);
    va_end(ap);
    return st;
}

sm_status cuda_fail(cudaError_t e, const char *what)
{
    if (e == cudaErrorMemoryAllocation) return fail(SM_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
    return fail(SM_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define LF_CUDA(expr, what)                           \
    do {                                              \
        cudaError_t e_ = (expr);                      \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

#define LF_LAUNCHED(what)                                   \
    do {                                                    \
        cudaError_t e_ = cudaGetLastError();                \
        if (e_ != cudaSuccess) return cuda_fail(e_, what);  \
    } while (0)

// Makes the mesh's device current for the duration of a call.
struct DeviceGuard {
    int prev = -1;
    bool changed = false;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) {
            changed = cudaSetDevice(dev) == cudaSuccess;
        }
    }
    ~DeviceGuard()
    {
        if (changed) cudaSetDevice(prev);
    }
};

// NVTX domain of the library: every launch scope below is a range named after
// its kernel kind, so that a timeline (nsys) or a filtered capture (ncu
// --nvtx) can pick the hot path's steps out; without a profiler attached the
// calls return at once.
nvtxDomainHandle_t nvtx_domain()
{
    static const nvtxDomainHandle_t d = nvtxDomainCreateA("labelfuse");
    return d;
}

const char *kernel_kind_name(int k)
{
    static const char *const names[SM_K_COUNT_KINDS] = {"project", "raster", "resolve", "count", "scatter",
                                                        "normalise", "render", "queue", "conf"};
    return k >= 0 && k < SM_K_COUNT_KINDS ? names[k] : "kernel";
}

// CUDA-event bracket of one launch when kernel timing is enabled, and an NVTX
// range around it always.
struct ProfScope {
    sm_mesh *m;
    int k;
    cudaStream_t s;
    sm_mesh::EvPair *ev = nullptr;
    // kernels: how many kernel launches the scope brackets
    ProfScope(sm_mesh *m_, sm_kernel k_, cudaStream_t s_, int kernels = 1) : m(m_), k((int)k_), s(s_)
    {
        nvtxEventAttributes_t a{};
        a.version = NVTX_VERSION;
        a.size = NVTX_EVENT_ATTRIB_STRUCT_SIZE;
        a.messageType = NVTX_MESSAGE_TYPE_ASCII;
        a.message.ascii = kernel_kind_name(k);
        nvtxDomainRangePushEx(nvtx_domain(), &a);
        if (!m->prof) return;
        m->ev_kernels[k] += kernels;
        if (m->ev_used[k] == m->ev[k].size()) {
            sm_mesh::EvPair p;
            if (cudaEventCreate(&p.a) != cudaSuccess) return;
            if (cudaEventCreate(&p.b) != cudaSuccess) {
                cudaEventDestroy(p.a);
                return;
            }
            m->ev[k].push_back(p);
        }
        ev = &m->ev[k][m->ev_used[k]++];
        cudaEventRecord(ev->a, s);
    }
    ~ProfScope()
    {
        if (ev) cudaEventRecord(ev->b, s);
        nvtxDomainRangePop(nvtx_domain());
    }
};

// Test hook (host only): with LABELFUSE_TEST_FAIL_ALLOC set, every device
// allocation of the library fails as if the device were out of memory, so
// the SM_ERR_OOM paths can be exercised without exhausting a GPU.
bool injected_alloc_failure() { return getenv("LABELFUSE_TEST_FAIL_ALLOC") != nullptr; }

cudaError_t device_alloc(void **p, size_t bytes)
{
    if (injected_alloc_failure()) return cudaErrorMemoryAllocation;
    return cudaMalloc(p, bytes);
}

// Compressible device memory (the GPU's compute data compression) for
// buffers that hold long runs of equal values.  Between two uses of a z-buffer
// slot its keys are re-armed to all-ones and written back to DRAM, and the
// next raster's atomics read them back: two transfers of constant data per
// pixel and use, which the memory system stores compressed in compressible
// memory; row maps, label images and the mostly-zero per-frame row histograms
// compress as well.  The allocation goes through the driver's virtual-memory
// calls (cuMemCreate with generic compression, then reserve, map and grant
// access), fetched from the runtime at run time so that the library has no
// link-time dependency on the driver library.  Where the device or driver
// offers no compression (or with LABELFUSE_COMPRESSIBLE_MEMORY=0 in the
// environment) these buffers are ordinary device memory.
struct VmmApi {
    decltype(&cuDeviceGet) device_get = nullptr;
    decltype(&cuDeviceGetAttribute) device_attr = nullptr;
    decltype(&cuMemGetAllocationGranularity) granularity = nullptr;
    decltype(&cuMemCreate) create = nullptr;
    decltype(&cuMemGetAllocationPropertiesFromHandle) props = nullptr;
    decltype(&cuMemAddressReserve) reserve = nullptr;
    decltype(&cuMemMap) map = nullptr;
    decltype(&cuMemSetAccess) access = nullptr;
    decltype(&cuMemUnmap) unmap = nullptr;
    decltype(&cuMemAddressFree) addr_free = nullptr;
    decltype(&cuMemRelease) release = nullptr;
    bool ok = false;
};

const VmmApi &vmm_api()
{
    static const VmmApi api = [] {
        VmmApi a;
        auto get = [](const char *name, void **fn) {
            cudaDriverEntryPointQueryResult q{};
            if (cudaGetDriverEntryPointByVersion(name, fn, CUDA_VERSION, cudaEnableDefault, &q) != cudaSuccess ||
                q != cudaDriverEntryPointSuccess) {
                cudaGetLastError();
                *fn = nullptr;
                return false;
            }
            return *fn != nullptr;
        };
        a.ok = get("cuDeviceGet", (void **)&a.device_get) && get("cuDeviceGetAttribute", (void **)&a.device_attr) &&
               get("cuMemGetAllocationGranularity", (void **)&a.granularity) &&
               get("cuMemCreate", (void **)&a.create) &&
               get("cuMemGetAllocationPropertiesFromHandle", (void **)&a.props) &&
               get("cuMemAddressReserve", (void **)&a.reserve) && get("cuMemMap", (void **)&a.map) &&
               get("cuMemSetAccess", (void **)&a.access) && get("cuMemUnmap", (void **)&a.unmap) &&
               get("cuMemAddressFree", (void **)&a.addr_free) && get("cuMemRelease", (void **)&a.release);
        return a;
    }();
    return api;
}

bool compression_wanted()
{
    const char *v = getenv("LABELFUSE_COMPRESSIBLE_MEMORY");
    return !(v && v[0] == '0');
}

// Maps `bytes` (rounded up to the allocation granularity, returned in
// *mapped) of compressible memory on device `dev`; false, with nothing held,
// if compression is unavailable or not granted.
bool compressible_alloc(int dev, size_t bytes, void **ptr, size_t *mapped, unsigned long long *handle)
{
    const VmmApi &api = vmm_api();
    if (!api.ok || !compression_wanted() || injected_alloc_failure()) return false;
    CUdevice d;
    int supported = 0;
    if (api.device_get(&d, dev) != CUDA_SUCCESS ||
        api.device_attr(&supported, CU_DEVICE_ATTRIBUTE_GENERIC_COMPRESSION_SUPPORTED, d) != CUDA_SUCCESS ||
        !supported)
        return false;
    CUmemAllocationProp prop;
    memset(&prop, 0, sizeof prop);
    prop.type = CU_MEM_ALLOCATION_TYPE_PINNED;
    prop.location.type = CU_MEM_LOCATION_TYPE_DEVICE;
    prop.location.id = d;
    prop.allocFlags.compressionType = CU_MEM_ALLOCATION_COMP_GENERIC;
    size_t gran = 0;
    if (api.granularity(&gran, &prop, CU_MEM_ALLOC_GRANULARITY_RECOMMENDED) != CUDA_SUCCESS || gran == 0) return false;
    const size_t size = (bytes + gran - 1) / gran * gran;
    CUmemGenericAllocationHandle h;
    if (api.create(&h, size, &prop, 0) != CUDA_SUCCESS) return false;
    CUmemAllocationProp got;
    memset(&got, 0, sizeof got);
    if (api.props(&got, h) != CUDA_SUCCESS || got.allocFlags.compressionType != CU_MEM_ALLOCATION_COMP_GENERIC) {
        api.release(h);
        return false;
    }
    CUdeviceptr va = 0;
    if (api.reserve(&va, size, gran, 0, 0) != CUDA_SUCCESS) {
        api.release(h);
        return false;
    }
    CUmemAccessDesc acc;
    memset(&acc, 0, sizeof acc);
    acc.location = prop.location;
    acc.flags = CU_MEM_ACCESS_FLAGS_PROT_READWRITE;
    if (api.map(va, size, 0, h, 0) != CUDA_SUCCESS) {
        api.addr_free(va, size);
        api.release(h);
        return false;
    }
    if (api.access(va, size, &acc, 1) != CUDA_SUCCESS) {
        api.unmap(va, size);
        api.addr_free(va, size);
        api.release(h);
        return false;
    }
    *ptr = reinterpret_cast<void *>(va);
    *mapped = size;
    *handle = (unsigned long long)h;
    return true;
}

// Releases a block of compressible_alloc; no work on the device may still use it.
void compressible_free(void *ptr, size_t mapped, unsigned long long handle)
{
    const VmmApi &api = vmm_api();
    const CUdeviceptr va = reinterpret_cast<CUdeviceptr>(ptr);
    api.unmap(va, mapped);
    api.addr_free(va, mapped);
    api.release((CUmemGenericAllocationHandle)handle);
}

template <class T>
sm_status grow(T **buf, int64_t *cap, int64_t need, cudaStream_t s, int fill, const char *what)
{
    if (*cap >= need) return SM_OK;
    if (*buf) LF_CUDA(cudaFreeAsync(*buf, s), what);
    *buf = nullptr;
    *cap = 0;
    void *p = nullptr;
    if (injected_alloc_failure()) return cuda_fail(cudaErrorMemoryAllocation, what);
    LF_CUDA(cudaMallocAsync(&p, (size_t)need * sizeof(T), s), what);
    if (fill >= 0) LF_CUDA(cudaMemsetAsync(p, fill, (size_t)need * sizeof(T), s), what);
    *buf = static_cast<T *>(p);
    *cap = need;
    return SM_OK;
}

// Room for `need` elements in *buf, in compressible memory where the device
// offers it (compressible_alloc), else stream-ordered device memory; fill >= 0
// sets every byte.  The z-buffer (re-armed to all-ones between uses), the row
// maps and label images (runs of equal values) and the per-frame row
// histograms (mostly zero) compress.  A
// compressible block is released only once the device is idle; inside a
// stream capture, where that wait is not allowed, the old block is kept until
// the mesh is freed and the new one is stream-ordered memory.
template <typename T>
sm_status grow_compressible(sm_mesh *m, T **buf, int64_t *cap, sm_mesh::VmmBlock *blk, int64_t need, cudaStream_t s,
                            int fill, const char *what)
{
    if (*cap >= need) return SM_OK;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    LF_CUDA(cudaStreamIsCapturing(s, &cs), what);
    const bool capturing = cs != cudaStreamCaptureStatusNone;
    if (*buf) {
        if (!blk->p) {
            LF_CUDA(cudaFreeAsync(*buf, s), what);
        } else if (capturing) {
            m->retired.push_back(*blk);
        } else {
            LF_CUDA(cudaDeviceSynchronize(), what);
            compressible_free(blk->p, blk->mapped, blk->handle);
        }
    }
    *buf = nullptr;
    *cap = 0;
    *blk = sm_mesh::VmmBlock{};
    const size_t bytes = (size_t)need * sizeof(T);
    void *p = nullptr;
    size_t mapped = 0;
    unsigned long long h = 0;
    if (!capturing && compressible_alloc(m->device, bytes, &p, &mapped, &h)) {
        *blk = sm_mesh::VmmBlock{p, mapped, h};
    } else {
        if (injected_alloc_failure()) return cuda_fail(cudaErrorMemoryAllocation, what);
        LF_CUDA(cudaMallocAsync(&p, bytes, s), what);
    }
    *buf = static_cast<T *>(p);
    *cap = need;
    if (fill >= 0) LF_CUDA(cudaMemsetAsync(p, fill, bytes, s), what);
    return SM_OK;
}

size_t dtype_size(sm_dtype d) { return d == SM_F32 ? 4 : (d == SM_BF16 ? 2 : 1); }

// Frames per batch: a batch's 64-bit z-buffers take up to ~48 MB (20 frames
// of 640 x 480) unless the autotuner chose another length.  Longer batches keep the mostly-culled raster launches and
// the streaming scatter launches long enough to fill the GPU, which matters
// more than keeping both z-buffer slots in L2; the per-frame row histograms
// of the image weights stay within ~512 MB.
// Most frames per launch pair: each pair costs about 36 us of pipeline fill
// and drain, so longer launches pay even when a batch's z-buffers leave L2.
constexpr int kMaxLaunchFrames = 1024;

int batch_frames(const sm_mesh *m, int64_t npix, int N, bool tuned = true)
{
    int64_t B = (tuned && m->tuned_B > 0 && m->tuned_npix == npix) ? m->tuned_B : (int64_t)(48u << 20) / (npix * 8);
    if (m->weight == SM_WEIGHT_IMAGE && m->n_x > 0) {
        const int64_t Bi = (int64_t)(512u << 20) / (m->n_x * 4);
        if (Bi < B) B = Bi;
    }
    if (B < 1) B = 1;
    if (B > kMaxLaunchFrames) B = kMaxLaunchFrames;
    // multiples of 4 frames keep every batch's probability, scale and row-map
    // base 16-byte aligned for the bulk copies (4 H W c bytes is a multiple
    // of 16 for c % 4 == 0)
    B = (B < 4) ? 4 : (B & ~3LL);
    if (B > N) B = N;
    return (int)B;
}

sm_status check_image(int32_t N, int32_t H, int32_t W)
{
    if (N < 0) return fail(SM_ERR_INVALID_ARG, "N = %d < 0", N);
    if (H < 1 || H > SM_MAX_IMAGE_DIM || W < 1 || W > SM_MAX_IMAGE_DIM)
        return fail(SM_ERR_INVALID_ARG, "image size %d x %d outside [1, %d]", H, W, SM_MAX_IMAGE_DIM);
    return SM_OK;
}

// Raster of frames [f0, f0 + nb) into the z-buffer keys (nb x H x W).
sm_status raster_only(sm_mesh *m, int f0, int nb, int H, int W, unsigned long long *keys, cudaStream_t s)
{
    const int64_t ncl = (m->F + lf::kClusterFaces - 1) / lf::kClusterFaces;
    sm_status st;
    if ((st = grow(&m->clist, &m->clist_cap, (int64_t)nb * ncl, s, -1, "cluster lists")) != SM_OK) return st;
    if ((st = grow(&m->ccount, &m->ccount_cap, (int64_t)nb, s, -1, "cluster counts")) != SM_OK) return st;
    {
        ProfScope p(m, SM_K_RASTER, s, 2);
        lf::launch_raster(m->verts, m->faces, m->F, m->bounds, m->cams, f0, nb, H, W, keys, m->clist, m->ccount, s);
    }
    LF_LAUNCHED("raster");
    return SM_OK;
}

// z-buffer keys -> row map (re-arms the keys).
sm_status resolve_only(sm_mesh *m, int f0, int nb, int H, int W, unsigned long long *keys, int32_t *idm,
                       cudaStream_t s, int32_t *idm2 = nullptr)
{
    {
        ProfScope p(m, SM_K_RESOLVE, s);
        lf::launch_resolve(keys, nb, H, W, m->texel_mode ? m->row0 : nullptr, m->texinfo, m->verts, m->faces,
                           m->cams, f0, idm, idm2, s);
    }
    LF_LAUNCHED("resolve");
    return SM_OK;
}

// Raster + resolve of frames [f0, f0 + nb) into idm (nb x H x W), one stream.
sm_status raster_batch(sm_mesh *m, int f0, int nb, int H, int W, int32_t *idm, cudaStream_t s)
{
    sm_status st = raster_only(m, f0, nb, H, W, m->keys, s);
    if (st != SM_OK) return st;
    return resolve_only(m, f0, nb, H, W, m->keys, idm, s);
}

// Elements per z-buffer slot, rounded so every slot starts 256-byte aligned.
int64_t slot_stride(int B, int64_t npix) { return ((int64_t)B * npix + 31) & ~31LL; }

// Cameras of N frames (set up on the device) and z-buffer room for `slots`
// slots of B frames; every key is empty between calls.
sm_status prepare_frames(sm_mesh *m, const sm_intrinsics *d_K, const double *d_T, int N, int64_t npix, int B,
                         bool need_idbuf, cudaStream_t s, int slots = 2)
{
    sm_status st;
    if ((st = grow(&m->cams, &m->cams_cap, N, s, -1, "camera buffer")) != SM_OK) return st;
    // (two slots for the stream path: raster of batch b+1 beside the scatter of batch b)
    if ((st = grow_compressible(m, &m->keys, &m->keys_cap, &m->keys_blk, slots * slot_stride(B, npix), s, 0xFF,
                                "z-buffer")) != SM_OK)
        return st;
    if (need_idbuf && (st = grow_compressible(m, &m->idbuf, &m->idbuf_cap, &m->idbuf_blk, (int64_t)B * npix, s, -1,
                                              "row-map buffer")) != SM_OK)
        return st;
    {
        ProfScope p(m, SM_K_PROJECT, s);
        lf::launch_project(d_K, d_T, N, m->cams, s);
    }
    LF_LAUNCHED("camera set-up");
    return SM_OK;
}

// Shape of the work-queue fusion for frames of npix pixels: the tuned or set
// shape, else defaults (32-frame batches, raster two batches ahead, one cull
// round per raster item, 128 tiles per scatter item: the fastest measured on
// the paper-shaped workload).
struct QueueShape {
    int B, L, R, S;
};

QueueShape queue_shape(const sm_mesh *m, int64_t npix)
{
    QueueShape q{32, 2, 1, 128};
    if (m->q_npix == npix) {
        if (m->qB > 0) q.B = m->qB;
        if (m->qL > 0) q.L = m->qL;
        if (m->qR > 0) q.R = m->qR;
        if (m->qS > 0) q.S = m->qS;
    }
    return q;
}

// One scene's pieces for work-queue launches: cameras set up and z-buffer
// slots grown; the full batches in pieces of at most fuse_queue_max_batches()
// batches, then the remaining frames (fewer than a batch) as one more piece.
struct QueuePrep {
    std::vector<lf::FuseQueueScene> full, rest;
    int lookahead = 1;
};

sm_status prepare_queue_scene(sm_mesh *m, const void *d_probs, sm_dtype dtype, const float *d_scale,
                              const sm_intrinsics *d_K, const double *d_T, int32_t N, int32_t H, int32_t W,
                              int32_t *d_idmap_out, cudaStream_t s, QueuePrep *out)
{
    const int64_t npix = (int64_t)H * W;
    const QueueShape qs = queue_shape(m, npix);
    const int B = N < qs.B ? N : qs.B;  // a multiple of 4 unless it is the whole call
    const int slots = qs.L + 2;
    const int nfull = N / B, rem = N - nfull * B;
    sm_status st;
    if ((st = prepare_frames(m, d_K, d_T, N, npix, B, false, s, slots)) != SM_OK) return st;
    if ((st = grow(&m->qctr, &m->qctr_cap, (int64_t)lf::fuse_queue_counter_words(lf::fuse_queue_max_batches()), s,
                   -1, "queue counters")) != SM_OK)
        return st;
    const size_t esz = dtype_size(dtype);
    lf::FuseQueueScene l{};
    l.V = m->verts;
    l.faces = m->faces;
    l.F = m->F;
    l.bounds = m->bounds;
    l.H = H;
    l.W = W;
    l.npix = npix;
    l.acc = m->acc;
    l.cnt = m->cnt;
    l.n_x = m->n_x;
    l.err = m->err;
    l.keys = m->keys;
    l.slot_stride = slot_stride(B, npix);
    l.slots = slots;
    l.raster_rounds = qs.R;
    l.scatter_tiles = qs.S;
    l.owner = m;
    auto piece = [&](int f0, int nb, int Bp) {
        lf::FuseQueueScene p = l;
        p.nb = nb;
        p.B = Bp;
        p.cams = m->cams + f0;
        p.probs = static_cast<const char *>(d_probs) + (size_t)f0 * npix * m->c * esz;
        p.scale = d_scale ? d_scale + (size_t)f0 * npix : nullptr;
        p.ids_out = d_idmap_out ? d_idmap_out + (int64_t)f0 * npix : nullptr;
        return p;
    };
    const int maxb = lf::fuse_queue_max_batches();
    for (int b0 = 0; b0 < nfull; b0 += maxb)
        out->full.push_back(piece(b0 * B, nfull - b0 < maxb ? nfull - b0 : maxb, B));
    if (rem > 0) out->rest.push_back(piece(nfull * B, 1, rem));
    out->lookahead = qs.L;
    m->normalised = false;
    return SM_OK;
}

// Launches the pieces in order, packed into as few work-queue launches as
// the limits allow (scenes and batches per launch, no two pieces of one mesh
// in a launch); every launch takes the smallest lookahead of its pieces.
sm_status launch_pieces(const std::vector<lf::FuseQueueScene> &pieces, const std::vector<int> &lookahead,
                        sm_dtype dtype, int c, sm_rule rule, sm_mesh *lead, cudaStream_t s)
{
    const int maxs = lf::fuse_queue_max_scenes(), maxb = lf::fuse_queue_max_batches();
    size_t k = 0;
    while (k < pieces.size()) {
        std::vector<lf::FuseQueueScene> batch;
        int G = 0, L = 4;
        while (k < pieces.size() && (int)batch.size() < maxs && G + pieces[k].nb <= maxb) {
            bool dup = false;
            for (const auto &q : batch) dup = dup || q.owner == pieces[k].owner;
            if (dup) break;
            batch.push_back(pieces[k]);
            G += pieces[k].nb;
            if (lookahead[k] < L) L = lookahead[k];
            ++k;
        }
        bool ok;
        {
            ProfScope p(lead, SM_K_QUEUE, s);
            ok = lf::launch_fuse_queue(batch.data(), (int)batch.size(), dtype, c, rule, L, lead->qctr, s);
        }
        if (!ok) return fail(SM_ERR_INTERNAL, "work-queue launch refused its pieces (%d)", (int)batch.size());
        LF_LAUNCHED("fusion work queue");
    }
    return SM_OK;
}

// Fusion of N frames in face mode with pixel weights through the persistent
// work-queue kernel: the full batches (in launches of at most
// fuse_queue_max_batches() batches), then the remaining frames.
sm_status fuse_queue_impl(sm_mesh *m, const void *d_probs, sm_dtype dtype, const float *d_scale,
                          const sm_intrinsics *d_K, const double *d_T, int32_t N, int32_t H, int32_t W,
                          int32_t *d_idmap_out, cudaStream_t s)
{
    QueuePrep prep;
    sm_status st = prepare_queue_scene(m, d_probs, dtype, d_scale, d_K, d_T, N, H, W, d_idmap_out, s, &prep);
    if (st != SM_OK) return st;
    std::vector<lf::FuseQueueScene> pieces(prep.full);
    pieces.insert(pieces.end(), prep.rest.begin(), prep.rest.end());
    return launch_pieces(pieces, std::vector<int>(pieces.size(), prep.lookahead), dtype, m->c, m->rule, m, s);
}

// Fusion of N frames (sm_fuse_frames; d_weights: explicit per-pixel weights, or null).
// Fusion of N frames.  d_weights: explicit per-pixel weights (replace w^(I));
// d_conf: confidence-network parameters, the weights computed per batch from
// the batch's z-buffer before its scatter (copied to d_w_out if given).
sm_status fuse_impl(sm_mesh *m, const void *d_probs, sm_dtype dtype, const float *d_scale, const sm_intrinsics *d_K,
                    const double *d_cam_to_world, int32_t N, int32_t H, int32_t W, const float *d_weights,
                    int32_t *d_idmap_out, void *stream, const float *d_conf = nullptr, float *d_w_out = nullptr)
{
    if (!m) return fail(SM_ERR_INVALID_ARG, "mesh is NULL");
    sm_status st = check_image(N, H, W);
    if (st != SM_OK) return st;
    if ((int)dtype < 0 || (int)dtype > 2) return fail(SM_ERR_INVALID_ARG, "unknown dtype %d", (int)dtype);
    if (dtype == SM_F32 && d_scale) return fail(SM_ERR_INVALID_ARG, "F32 probabilities take no scale");
    if (dtype != SM_F32 && !d_scale && N > 0) return fail(SM_ERR_INVALID_ARG, "BF16/FP8 need a per-pixel scale");
    if (N == 0) return SM_OK;
    if (!d_probs || !d_K || !d_cam_to_world) return fail(SM_ERR_INVALID_ARG, "NULL input pointer");
    if (((uintptr_t)d_probs & 15) != 0) return fail(SM_ERR_INVALID_ARG, "probabilities not 16-byte aligned");
    DeviceGuard g(m->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t npix = (int64_t)H * W;
    const int B = batch_frames(m, npix, N);
    const bool image_w = m->weight == SM_WEIGHT_IMAGE && !d_weights && !d_conf;  // explicit weights replace w^(I)
    const bool tma = lf::scatter_tma_supported(m->c);
    // face mode with the pipelined scatter: the scatter reads the z-buffer
    // keys itself; otherwise a resolve pass writes the row map first
    const bool from_keys = tma && !m->texel_mode;
    // face mode with pixel weights and c = 20 / 40: raster and scatter of the
    // whole call in the persistent work-queue kernel
    if (from_keys && !image_w && !d_weights && !d_conf && lf::fuse_queue_supported(m->c) && m->use_queue)
        return fuse_queue_impl(m, d_probs, dtype, d_scale, d_K, d_cam_to_world, N, H, W, d_idmap_out, s);
    const bool need_ids = !from_keys || image_w;
    // the pipelined scatter reads its row map from the library's aligned buffer
    const bool ids_internal = need_ids && (!d_idmap_out || (tma && !from_keys));
    if ((st = prepare_frames(m, d_K, d_cam_to_world, N, npix, B, ids_internal, s)) != SM_OK) return st;
    if (image_w && (st = grow_compressible(m, &m->fcnt, &m->fcnt_cap, &m->fcnt_blk, (int64_t)B * m->n_x, s, 0,
                                           "row histograms")) != SM_OK)
        return st;
    if (d_conf && (st = grow(&m->wbuf, &m->wbuf_cap, (int64_t)B * npix, s, -1, "confidence weights")) != SM_OK)
        return st;
    const size_t esz = dtype_size(dtype);
    cudaStream_t r = m->rstream;
    LF_CUDA(cudaEventRecord(m->ev_start, s), "event");
    LF_CUDA(cudaStreamWaitEvent(r, m->ev_start, 0), "event");
    for (int b = 0, f0 = 0; f0 < N; ++b, f0 += B) {
        const int nb = (N - f0 < B) ? N - f0 : B;
        const int slot = b & 1;
        unsigned long long *keys = m->keys + (int64_t)slot * slot_stride(B, npix);
        int32_t *user_idm = d_idmap_out ? d_idmap_out + (int64_t)f0 * npix : nullptr;
        int32_t *idm = ids_internal ? m->idbuf : user_idm;
        // raster of this batch on the raster stream, once the scatter that
        // last used this z-buffer slot has re-armed it
        if (b >= 2) LF_CUDA(cudaStreamWaitEvent(r, m->ev_scat[slot], 0), "event");
        if ((st = raster_only(m, f0, nb, H, W, keys, r)) != SM_OK) return st;
        LF_CUDA(cudaEventRecord(m->ev_rast[slot], r), "event");
        LF_CUDA(cudaStreamWaitEvent(s, m->ev_rast[slot], 0), "event");
        if (d_conf) {
            // weights from the keys as they stand (the scatter or the resolve
            // re-arms them afterwards)
            {
                ProfScope p(m, SM_K_CONF, s);
                lf::launch_conf_weights(keys, npix * nb, H, W, m->verts, m->faces, m->F, d_K + f0,
                                        d_cam_to_world + 16 * (int64_t)f0,
                                        static_cast<const char *>(d_probs) + (size_t)f0 * npix * m->c * esz, dtype,
                                        d_scale ? d_scale + (size_t)f0 * npix : nullptr, m->c, d_conf, m->wbuf,
                                        nullptr, s);
            }
            LF_LAUNCHED("confidence weights");
            if (d_w_out)
                LF_CUDA(cudaMemcpyAsync(d_w_out + (size_t)f0 * npix, m->wbuf, (size_t)nb * npix * sizeof(float),
                                        cudaMemcpyDeviceToDevice, s),
                        "weights copy");
        }
        if (!from_keys &&
            (st = resolve_only(m, f0, nb, H, W, keys, idm, s, idm != user_idm ? user_idm : nullptr)) != SM_OK)
            return st;
        if (image_w) {
            ProfScope p(m, SM_K_COUNT, s);
            lf::launch_count(from_keys ? nullptr : idm, keys, npix, nb, m->fcnt, m->n_x, s);
        }
        {
            ProfScope p(m, SM_K_SCATTER, s);
            const char *probs = static_cast<const char *>(d_probs) + (size_t)f0 * npix * m->c * esz;
            const float *scale = d_scale ? d_scale + (size_t)f0 * npix : nullptr;
            const uint32_t *fcnt = image_w ? m->fcnt : nullptr;
            const float *wpix = d_conf ? m->wbuf : d_weights ? d_weights + (size_t)f0 * npix : nullptr;
            if (tma)
                lf::launch_scatter_tma(m->rule, dtype, probs, scale, from_keys ? keys : nullptr,
                                       from_keys ? nullptr : idm, from_keys ? idm : nullptr, npix * nb, npix, m->c,
                                       fcnt, m->alpha, wpix, m->n_x, m->acc, m->cnt, m->err, s);
            else
                lf::launch_scatter(m->rule, dtype, probs, scale, idm, npix, nb, m->c, fcnt, m->alpha, wpix, m->n_x,
                                   m->acc, m->cnt, m->err, s);
        }
        LF_LAUNCHED("scatter");
        if (image_w) {
            ProfScope p(m, SM_K_COUNT, s);
            lf::launch_count_reset(idm, npix, nb, m->fcnt, m->n_x, s);
        }
        LF_LAUNCHED("histogram reset");
        LF_CUDA(cudaEventRecord(m->ev_scat[slot], s), "event");
    }
    m->normalised = false;
    return SM_OK;
}
}  // namespace

extern "C" {

const char *sm_status_string(sm_status s)
{
    switch (s) {
    case SM_OK: return "ok";
    case SM_ERR_INVALID_ARG: return "invalid argument";
    case SM_ERR_OOM: return "out of device memory";
    case SM_ERR_CUDA: return "CUDA error";
    case SM_ERR_STATE: return "invalid state";
    case SM_ERR_TIMEOUT: return "timeout";
    case SM_ERR_INTERNAL: return "error latched by a kernel";
    }
    return "unknown status";
}

const char *sm_last_error(void) { return g_last_error; }

sm_status sm_mesh_upload(const float *d_vertices, int64_t V, const int32_t *d_faces, int64_t F,
                         const int32_t *d_texel_res, int32_t n_classes, sm_rule rule, sm_weight weight,
                         void *stream, sm_mesh **out)
{
    if (!out) return fail(SM_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (V < 0 || F < 0) return fail(SM_ERR_INVALID_ARG, "negative V or F");
    if (F > 0 && (!d_vertices || !d_faces)) return fail(SM_ERR_INVALID_ARG, "vertices/faces NULL");
    if (V >= (1LL << 31) || F >= (1LL << 31)) return fail(SM_ERR_INVALID_ARG, "V or F >= 2^31");
    if (n_classes < 1 || n_classes > SM_MAX_CLASSES)
        return fail(SM_ERR_INVALID_ARG, "n_classes = %d outside [1, %d]", n_classes, SM_MAX_CLASSES);
    if ((int)rule < 0 || (int)rule > 3) return fail(SM_ERR_INVALID_ARG, "unknown rule %d", (int)rule);
    if ((int)weight < 0 || (int)weight > 1) return fail(SM_ERR_INVALID_ARG, "unknown weight %d", (int)weight);
    cudaStream_t s = static_cast<cudaStream_t>(stream);

    sm_mesh *m = new (std::nothrow) sm_mesh();
    if (!m) return fail(SM_ERR_OOM, "host allocation");
    auto bail = [&](sm_status st) {
        sm_mesh_free(m);
        return st;
    };
    if (cudaGetDevice(&m->device) != cudaSuccess) return bail(fail(SM_ERR_CUDA, "no current CUDA device"));
    m->V = V;
    m->F = F;
    m->c = n_classes;
    m->rule = rule;
    m->weight = weight;
    m->texel_mode = d_texel_res != nullptr;

    cudaError_t e;
    if ((e = device_alloc((void **)&m->err, 2 * sizeof(int32_t))) != cudaSuccess) return bail(cuda_fail(e, "error latch"));
    if ((e = cudaMemsetAsync(m->err, 0, 2 * sizeof(int32_t), s)) != cudaSuccess) return bail(cuda_fail(e, "memset"));
    if ((e = device_alloc((void **)&m->verts, (size_t)(V > 0 ? V : 1) * sizeof(float4))) != cudaSuccess)
        return bail(cuda_fail(e, "vertex buffer"));
    if ((e = device_alloc((void **)&m->faces, (size_t)(F > 0 ? F : 1) * sizeof(int4))) != cudaSuccess)
        return bail(cuda_fail(e, "face buffer"));
    const int64_t nclusters = (F + lf::kClusterFaces - 1) / lf::kClusterFaces;
    if ((e = device_alloc((void **)&m->bounds, (size_t)(nclusters > 0 ? 2 * nclusters : 2) * sizeof(float4))) != cudaSuccess)
        return bail(cuda_fail(e, "cluster bounds"));
    if ((e = cudaStreamCreateWithFlags(&m->rstream, cudaStreamNonBlocking)) != cudaSuccess)
        return bail(cuda_fail(e, "raster stream"));
    if ((e = cudaEventCreateWithFlags(&m->ev_start, cudaEventDisableTiming)) != cudaSuccess)
        return bail(cuda_fail(e, "events"));
    for (cudaStream_t &cs : m->cstream)
        if ((e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking)) != cudaSuccess)
            return bail(cuda_fail(e, "copy stream"));
    for (int k = 0; k < 2; ++k) {
        cudaEvent_t *evs[] = {&m->ev_rast[k], &m->ev_scat[k], &m->ev_free[k]};
        for (cudaEvent_t *ev : evs)
            if ((e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming)) != cudaSuccess)
                return bail(cuda_fail(e, "events"));
        for (cudaEvent_t &ev : m->ev_h2d[k])
            if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess)
                return bail(cuda_fail(e, "events"));
    }
    lf::launch_pack_mesh(d_vertices, V, d_faces, F, m->verts, m->faces, m->err, s);
    if ((e = cudaGetLastError()) != cudaSuccess) return bail(cuda_fail(e, "pack mesh"));
    lf::launch_cluster_bounds(m->verts, m->faces, F, m->bounds, s);
    if ((e = cudaGetLastError()) != cudaSuccess) return bail(cuda_fail(e, "cluster bounds"));

    int64_t n_x = F;
    if (m->texel_mode) {
        if ((e = device_alloc((void **)&m->row0, (size_t)(F > 0 ? F : 1) * sizeof(int32_t))) != cudaSuccess)
            return bail(cuda_fail(e, "row offsets"));
        if ((e = device_alloc((void **)&m->texinfo, (size_t)(F > 0 ? F : 1) * sizeof(int32_t))) != cudaSuccess)
            return bail(cuda_fail(e, "texel info"));
        void *scratch = nullptr;
        int64_t *d_nx = nullptr;
        if ((e = device_alloc(&scratch, lf::texel_scan_scratch_bytes(F))) != cudaSuccess)
            return bail(cuda_fail(e, "scan scratch"));
        if ((e = device_alloc((void **)&d_nx, sizeof(int64_t))) != cudaSuccess) {
            cudaFree(scratch);
            return bail(cuda_fail(e, "scan scratch"));
        }
        lf::launch_texel_layout(d_texel_res, m->verts, m->faces, F, m->texinfo, m->row0, d_nx, scratch, m->err, s);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(&n_x, d_nx, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        cudaFree(scratch);
        cudaFree(d_nx);
        if (e != cudaSuccess) return bail(cuda_fail(e, "texel layout"));
    }
    int32_t latched = 0;
    if ((e = cudaMemcpyAsync(&latched, m->err, sizeof(int32_t), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
        return bail(cuda_fail(e, "read error latch"));
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return bail(cuda_fail(e, "upload"));
    if (latched == lf::kErrTexelRes)
        return bail(fail(SM_ERR_INVALID_ARG, "texel steps outside [1, %d]", SM_MAX_TEXEL_RES));
    if (latched == lf::kErrRowOverflow || n_x >= (1LL << 31))
        return bail(fail(SM_ERR_INVALID_ARG, "n_x = %lld texel rows >= 2^31", (long long)n_x));
    m->n_x = n_x;

    const size_t acc_bytes = (size_t)(n_x > 0 ? n_x : 1) * n_classes * sizeof(float);
    if ((e = device_alloc((void **)&m->acc, acc_bytes)) != cudaSuccess) return bail(cuda_fail(e, "accumulators"));
    if ((e = device_alloc((void **)&m->cnt, (size_t)(n_x > 0 ? n_x : 1) * sizeof(uint32_t))) != cudaSuccess)
        return bail(cuda_fail(e, "counts"));
    if ((e = device_alloc((void **)&m->labels8, (size_t)(n_x > 0 ? n_x : 1))) != cudaSuccess)
        return bail(cuda_fail(e, "labels"));
    if ((e = cudaMemsetAsync(m->acc, 0, acc_bytes, s)) != cudaSuccess) return bail(cuda_fail(e, "memset"));
    if ((e = cudaMemsetAsync(m->cnt, 0, (size_t)(n_x > 0 ? n_x : 1) * sizeof(uint32_t), s)) != cudaSuccess)
        return bail(cuda_fail(e, "memset"));
    if ((e = cudaMemsetAsync(m->labels8, 0xFF, (size_t)(n_x > 0 ? n_x : 1), s)) != cudaSuccess)
        return bail(cuda_fail(e, "memset"));
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return bail(cuda_fail(e, "upload"));
    *out = m;
    return SM_OK;
}

sm_status sm_fuse_frames(sm_mesh *m, const void *d_probs, sm_dtype dtype, const float *d_scale,
                         const sm_intrinsics *d_K, const double *d_cam_to_world, int32_t N, int32_t H, int32_t W,
                         int32_t *d_idmap_out, void *stream)
{
    return fuse_impl(m, d_probs, dtype, d_scale, d_K, d_cam_to_world, N, H, W, nullptr, d_idmap_out, stream);
}

sm_status sm_fuse_frames_weighted(sm_mesh *m, const void *d_probs, sm_dtype dtype, const float *d_scale,
                                  const sm_intrinsics *d_K, const double *d_cam_to_world, int32_t N, int32_t H,
                                  int32_t W, const float *d_weights, int32_t *d_idmap_out, void *stream)
{
    if (N > 0 && !d_weights) return fail(SM_ERR_INVALID_ARG, "weights are NULL");
    return fuse_impl(m, d_probs, dtype, d_scale, d_K, d_cam_to_world, N, H, W, d_weights, d_idmap_out, stream);
}

sm_status sm_fuse_frames_confident(sm_mesh *m, const void *d_probs, sm_dtype dtype, const float *d_scale,
                                   const sm_intrinsics *d_K, const double *d_cam_to_world, int32_t N, int32_t H,
                                   int32_t W, const float *d_params, float *d_w_out, int32_t *d_idmap_out,
                                   void *stream)
{
    if (!d_params && N > 0) return fail(SM_ERR_INVALID_ARG, "NULL confidence parameters");
    return fuse_impl(m, d_probs, dtype, d_scale, d_K, d_cam_to_world, N, H, W, nullptr, d_idmap_out, stream, d_params,
                     d_w_out);
}

sm_status sm_fuse_scenes(const sm_scene_frames *scenes, int32_t n, void *stream)
{
    if (n < 0 || (n > 0 && !scenes)) return fail(SM_ERR_INVALID_ARG, "scenes is NULL or n < 0");
    if (n == 0) return SM_OK;
    for (int k = 0; k < n; ++k) {
        const sm_scene_frames &sf = scenes[k];
        if (!sf.mesh) return fail(SM_ERR_INVALID_ARG, "scene %d: mesh is NULL", k);
        for (int j = 0; j < k; ++j)
            if (scenes[j].mesh == sf.mesh) return fail(SM_ERR_INVALID_ARG, "scenes %d and %d share a mesh", j, k);
    }
    for (int k = 0; k < n; ++k) {
        const sm_scene_frames &sf = scenes[k];
        if (sf.mesh->device != scenes[0].mesh->device)
            return fail(SM_ERR_INVALID_ARG, "scene %d: its mesh is on device %d, scene 0's on %d", k, sf.mesh->device,
                        scenes[0].mesh->device);
        sm_status st = check_image(sf.N, sf.H, sf.W);
        if (st != SM_OK) {
            char msg[sizeof g_last_error];
            snprintf(msg, sizeof msg, "%s", g_last_error);
            return fail(st, "scene %d: %s", k, msg);
        }
        if ((int)sf.dtype < 0 || (int)sf.dtype > 2) return fail(SM_ERR_INVALID_ARG, "scene %d: unknown dtype", k);
        if ((sf.dtype == SM_F32) != (sf.d_scale == nullptr) && sf.N > 0)
            return fail(SM_ERR_INVALID_ARG, "scene %d: a scale is given iff BF16/FP8", k);
        if (sf.N > 0 && (!sf.d_probs || !sf.d_K || !sf.d_cam_to_world))
            return fail(SM_ERR_INVALID_ARG, "scene %d: NULL input pointer", k);
        if (sf.N > 0 && ((uintptr_t)sf.d_probs & 15) != 0)
            return fail(SM_ERR_INVALID_ARG, "scene %d: probabilities not 16-byte aligned", k);
    }
    DeviceGuard g(scenes[0].mesh->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // scenes the work queue applies to are grouped by (class count, storage
    // type, rule): one persistent launch (plus one for remainders) per group
    // of up to fuse_queue_max_scenes() scenes; the others fuse on their own
    bool done[1024] = {};
    if (n > 1024) return fail(SM_ERR_INVALID_ARG, "at most 1024 scenes per call (got %d)", n);
    for (int k = 0; k < n; ++k) {
        const sm_scene_frames &sf = scenes[k];
        sm_mesh *m = sf.mesh;
        const bool eligible = sf.N > 0 && !m->texel_mode && m->weight == SM_WEIGHT_PIXEL &&
                              lf::scatter_tma_supported(m->c) && lf::fuse_queue_supported(m->c);
        if (!eligible) {
            sm_status st = sm_fuse_frames(m, sf.d_probs, sf.dtype, sf.d_scale, sf.d_K, sf.d_cam_to_world, sf.N, sf.H,
                                          sf.W, sf.d_idmap_out, stream);
            if (st != SM_OK) return st;
            done[k] = true;
        }
    }
    for (int k = 0; k < n; ++k) {
        if (done[k]) continue;
        // the group of scene k: every not yet fused scene with its class
        // count, storage type and rule; their full-batch pieces first, then
        // the remainders, packed into work-queue launches
        std::vector<lf::FuseQueueScene> full, rest;
        std::vector<int> lfull, lrest;
        sm_mesh *lead = scenes[k].mesh;
        for (int j = k; j < n; ++j) {
            const sm_scene_frames &sf = scenes[j];
            if (done[j] || sf.mesh->c != lead->c || sf.dtype != scenes[k].dtype || sf.mesh->rule != lead->rule)
                continue;
            QueuePrep prep;
            sm_status st = prepare_queue_scene(sf.mesh, sf.d_probs, sf.dtype, sf.d_scale, sf.d_K, sf.d_cam_to_world,
                                               sf.N, sf.H, sf.W, sf.d_idmap_out, s, &prep);
            if (st != SM_OK) return st;
            full.insert(full.end(), prep.full.begin(), prep.full.end());
            lfull.insert(lfull.end(), prep.full.size(), prep.lookahead);
            rest.insert(rest.end(), prep.rest.begin(), prep.rest.end());
            lrest.insert(lrest.end(), prep.rest.size(), prep.lookahead);
            done[j] = true;
        }
        full.insert(full.end(), rest.begin(), rest.end());
        lfull.insert(lfull.end(), lrest.begin(), lrest.end());
        sm_status st = launch_pieces(full, lfull, scenes[k].dtype, lead->c, lead->rule, lead, s);
        if (st != SM_OK) return st;
    }
    return SM_OK;
}

sm_status sm_normalise(sm_mesh *m, float *d_dist, int32_t *d_labels, void *stream)
{
    if (!m) return fail(SM_ERR_INVALID_ARG, "mesh is NULL");
    DeviceGuard g(m->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    {
        ProfScope p(m, SM_K_NORMALISE, s);
        lf::launch_normalise(m->rule, m->acc, m->cnt, m->n_x, m->c, d_dist, d_labels, m->labels8, s);
    }
    LF_LAUNCHED("normalise");
    m->normalised = true;
    return SM_OK;
}

sm_status sm_render_labels(sm_mesh *m, const sm_intrinsics *d_K, const double *d_cam_to_world, int32_t N,
                           int32_t H, int32_t W, uint8_t *d_labels_out, int32_t *d_idmap_out, void *stream)
{
    if (!m) return fail(SM_ERR_INVALID_ARG, "mesh is NULL");
    sm_status st = check_image(N, H, W);
    if (st != SM_OK) return st;
    if (!m->normalised) return fail(SM_ERR_STATE, "sm_render_labels before sm_normalise");
    if (N == 0) return SM_OK;
    if (!d_K || !d_cam_to_world || !d_labels_out) return fail(SM_ERR_INVALID_ARG, "NULL pointer");
    DeviceGuard g(m->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t npix = (int64_t)H * W;
    const int B = batch_frames(m, npix, N);
    if ((st = prepare_frames(m, d_K, d_cam_to_world, N, npix, B, d_idmap_out == nullptr, s)) != SM_OK) return st;
    for (int f0 = 0; f0 < N; f0 += B) {
        const int nb = (N - f0 < B) ? N - f0 : B;
        int32_t *idm = d_idmap_out ? d_idmap_out + (int64_t)f0 * npix : m->idbuf;
        if ((st = raster_batch(m, f0, nb, H, W, idm, s)) != SM_OK) return st;
        {
            ProfScope p(m, SM_K_RENDER, s);
            lf::launch_render(idm, npix * nb, m->labels8, m->n_x, d_labels_out + (int64_t)f0 * npix, s);
        }
        LF_LAUNCHED("render");
    }
    return SM_OK;
}

sm_status sm_render_idmap(sm_mesh *m, const int32_t *d_idmap, int64_t n_pixels, uint8_t *d_labels_out,
                          void *stream)
{
    if (!m) return fail(SM_ERR_INVALID_ARG, "mesh is NULL");
    if (n_pixels < 0) return fail(SM_ERR_INVALID_ARG, "n_pixels < 0");
    if (!m->normalised) return fail(SM_ERR_STATE, "sm_render_idmap before sm_normalise");
    if (n_pixels == 0) return SM_OK;
    if (!d_idmap || !d_labels_out) return fail(SM_ERR_INVALID_ARG, "NULL pointer");
    DeviceGuard g(m->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    {
        ProfScope p(m, SM_K_RENDER, s);
        lf::launch_render(d_idmap, n_pixels, m->labels8, m->n_x, d_labels_out, s);
    }
    LF_LAUNCHED("render");
    return SM_OK;
}

sm_status sm_set_weight_mix(sm_mesh *m, float alpha)
{
    if (!m) return fail(SM_ERR_INVALID_ARG, "mesh is NULL");
    if (m->weight != SM_WEIGHT_IMAGE) return fail(SM_ERR_INVALID_ARG, "the weight mix needs a w^(I) mesh");
    if (!(alpha >= 0.0f && alpha <= 1.0f)) return fail(SM_ERR_INVALID_ARG, "alpha %g outside [0, 1]", (double)alpha);
    m->alpha = alpha;
    return SM_OK;
}

sm_status sm_texel_res_from_gamma(sm_mesh *m, const sm_intrinsics *d_K, const double *d_cam_to_world, int32_t N,
                                  int32_t H, int32_t W, float gamma, int32_t *d_area_out, int32_t *d_texel_res_out,
                                  void *stream)
{
    if (!m) return fail(SM_ERR_INVALID_ARG, "mesh is NULL");
    if (m->texel_mode) return fail(SM_ERR_STATE, "the visible-area pre-pass needs a mesh uploaded without texels");
    sm_status st = check_image(N, H, W);
    if (st != SM_OK) return st;
    if (!(gamma >= 0.0f && gamma <= 64.0f)) return fail(SM_ERR_INVALID_ARG, "gamma %g outside [0, 64]", (double)gamma);
    if (!d_texel_res_out || (N > 0 && (!d_K || !d_cam_to_world))) return fail(SM_ERR_INVALID_ARG, "NULL pointer");
    DeviceGuard g(m->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t F = m->F, npix = (int64_t)H * W;
    if ((st = grow(&m->area, &m->area_cap, F > 0 ? F : 1, s, -1, "area buffer")) != SM_OK) return st;
    LF_CUDA(cudaMemsetAsync(m->area, 0, (size_t)(F > 0 ? F : 1) * sizeof(int32_t), s), "area buffer");
    if (N > 0 && F > 0) {
        const int B = batch_frames(m, npix, N);
        if ((st = prepare_frames(m, d_K, d_cam_to_world, N, npix, B, false, s)) != SM_OK) return st;
        // per-frame counts share the w^(I) histogram buffer (zero between uses)
        if ((st = grow_compressible(m, &m->fcnt, &m->fcnt_cap, &m->fcnt_blk, (int64_t)B * F, s, 0,
                                    "per-frame counts")) != SM_OK)
            return st;
        for (int f0 = 0; f0 < N; f0 += B) {
            const int nb = (N - f0 < B) ? N - f0 : B;
            if ((st = raster_only(m, f0, nb, H, W, m->keys, s)) != SM_OK) return st;
            lf::launch_area_count(m->keys, npix, nb, m->fcnt, F, s);
            lf::launch_area_max(m->fcnt, nb, F, m->area, s);
            LF_LAUNCHED("visible-area pre-pass");
        }
    }
    lf::launch_texel_res(m->area, F, gamma, d_texel_res_out, s);
    LF_LAUNCHED("texel steps");
    if (d_area_out && F > 0)
        LF_CUDA(cudaMemcpyAsync(d_area_out, m->area, (size_t)F * sizeof(int32_t), cudaMemcpyDeviceToDevice, s),
                "copy areas");
    return SM_OK;
}

sm_status sm_autotune_batch(sm_mesh *m, const void *d_probs, sm_dtype dtype, const float *d_scale,
                            const sm_intrinsics *d_K, const double *d_cam_to_world, int32_t N, int32_t H, int32_t W,
                            int32_t *best_out, void *stream)
{
    if (!m) return fail(SM_ERR_INVALID_ARG, "mesh is NULL");
    sm_status st = check_image(N, H, W);
    if (st != SM_OK) return st;
    if (N < 4) return fail(SM_ERR_INVALID_ARG, "the autotuner needs at least 4 frames (got %d)", N);
    DeviceGuard g(m->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t npix = (int64_t)H * W;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    LF_CUDA(cudaEventCreate(&e0), "events");
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return fail(SM_ERR_CUDA, "events");
    }
    // time of one fusion of the first n frames per frame (two passes: the
    // first sizes the scratch buffers, the second is timed)
    auto per_frame = [&](int n, float *out) -> sm_status {
        float ms = 0.0f;
        sm_status r = SM_OK;
        for (int rep = 0; rep < 2 && r == SM_OK; ++rep) {
            if ((r = sm_reset(m, stream)) != SM_OK) break;
            if (cudaEventRecord(e0, s) != cudaSuccess) r = fail(SM_ERR_CUDA, "event");
            if (r == SM_OK) r = sm_fuse_frames(m, d_probs, dtype, d_scale, d_K, d_cam_to_world, n, H, W, nullptr, stream);
            if (r == SM_OK && cudaEventRecord(e1, s) != cudaSuccess) r = fail(SM_ERR_CUDA, "event");
            if (r == SM_OK && cudaEventSynchronize(e1) != cudaSuccess) r = fail(SM_ERR_CUDA, "synchronise");
            if (r == SM_OK) cudaEventElapsedTime(&ms, e0, e1);
        }
        *out = ms / (float)n;
        return r;
    };
    const bool eligible = !m->texel_mode && m->weight == SM_WEIGHT_PIXEL && lf::scatter_tma_supported(m->c) &&
                          lf::fuse_queue_supported(m->c);
    const bool saved_queue = m->use_queue;
    int best = 0;
    float best_stream = 0.0f, best_queue = 0.0f;
    {
        // two-stream path: frames per launch
        m->use_queue = false;
        const int saved_B = m->tuned_B;
        const int64_t saved_npix = m->tuned_npix;
        // candidates: multiples of 4 frames, spaced by about a quarter, whose two
        // z-buffer slots stay within 8 GB
        static const int kCandidates[] = {4,   8,   12,  16,  20,  24,  32,  40,  48,  64,  80,
                                          96,  128, 160, 192, 256, 320, 384, 512, 640, 768, 1024};
        for (const int B : kCandidates) {
            if (B > kMaxLaunchFrames || B > N || (int64_t)B * npix * 16 > (8192ll << 20)) break;
            m->tuned_B = B;
            m->tuned_npix = npix;
            float ms = 0.0f;
            if ((st = per_frame((N / B) * B, &ms)) != SM_OK) break;  // whole launches only
            if (best == 0 || ms < best_stream) {
                best = B;
                best_stream = ms;
            }
        }
        if (st != SM_OK || best == 0) {
            m->tuned_B = saved_B;
            m->tuned_npix = saved_npix;
        } else {
            m->tuned_B = best;
            m->tuned_npix = npix;
        }
    }
    if (eligible && st == SM_OK && best != 0) {
        // work-queue path: its shape, one parameter at a time from the
        // defaults (frames per batch, raster lookahead, cull rounds per raster
        // item, tiles per scatter item); kept if it beats the two-stream path
        const QueueShape saved{m->qB, m->qL, m->qR, m->qS};
        const int64_t saved_npix = m->q_npix;
        QueueShape cur = queue_shape(m, -1);
        m->q_npix = npix;
        m->use_queue = true;
        auto apply = [&](const QueueShape &q) {
            m->qB = q.B;
            m->qL = q.L;
            m->qR = q.R;
            m->qS = q.S;
        };
        apply(cur);
        st = per_frame(N, &best_queue);
        const int Bs[] = {8, 16, 24, 32, 48, 64}, Ls[] = {1, 2, 3}, Rs[] = {1, 2, 4}, Ss[] = {32, 64, 128, 256};
        for (int dim = 0; dim < 4 && st == SM_OK; ++dim) {
            const int *vals = dim == 0 ? Bs : dim == 1 ? Ls : dim == 2 ? Rs : Ss;
            const int nv = dim == 0 ? 6 : dim == 1 ? 3 : dim == 2 ? 3 : 4;
            for (int k = 0; k < nv && st == SM_OK; ++k) {
                QueueShape c = cur;
                int *field = dim == 0 ? &c.B : dim == 1 ? &c.L : dim == 2 ? &c.R : &c.S;
                if (*field == vals[k] || (dim == 0 && vals[k] > N)) continue;
                *field = vals[k];
                apply(c);
                float ms = 0.0f;
                if ((st = per_frame(N, &ms)) != SM_OK) break;
                if (ms < best_queue) {
                    best_queue = ms;
                    cur = c;
                }
            }
        }
        if (st == SM_OK && best_queue < best_stream) {
            apply(cur);
            best = cur.B;
        } else {
            apply(saved);
            m->q_npix = saved_npix;
            m->use_queue = false;
        }
    } else {
        m->use_queue = saved_queue;  // the queue path does not apply to this mesh (or tuning failed)
    }
    if (st == SM_OK) st = sm_reset(m, stream);
    if (st != SM_OK) m->use_queue = saved_queue;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != SM_OK) return st;
    if (best == 0) return fail(SM_ERR_INTERNAL, "autotuner found no candidate");
    if (best_out) *best_out = best;
    return SM_OK;
}

sm_status sm_set_launch_frames(sm_mesh *m, int32_t H, int32_t W, int32_t frames)
{
    if (!m) return fail(SM_ERR_INVALID_ARG, "mesh is NULL");
    sm_status st = check_image(0, H, W);
    if (st != SM_OK) return st;
    if (frames < 0 || frames > kMaxLaunchFrames || (frames & 3) != 0)
        return fail(SM_ERR_INVALID_ARG, "frames per launch %d: a multiple of 4 in [4, %d], or 0", frames,
                    kMaxLaunchFrames);
    m->tuned_B = frames;
    m->tuned_npix = frames ? (int64_t)H * W : 0;
    return SM_OK;
}

sm_status sm_set_queue_shape(sm_mesh *m, int32_t H, int32_t W, int32_t frames_per_batch, int32_t lookahead,
                             int32_t raster_rounds, int32_t scatter_tiles)
{
    if (!m) return fail(SM_ERR_INVALID_ARG, "mesh is NULL");
    sm_status st = check_image(0, H, W);
    if (st != SM_OK) return st;
    if (frames_per_batch == 0) {
        m->use_queue = false;
        return SM_OK;
    }
    if (frames_per_batch < 4 || frames_per_batch > 128 || (frames_per_batch & 3) != 0)
        return fail(SM_ERR_INVALID_ARG, "frames per batch %d: a multiple of 4 in [4, 128], or 0", frames_per_batch);
    if (lookahead < 1 || lookahead > 4) return fail(SM_ERR_INVALID_ARG, "lookahead %d outside [1, 4]", lookahead);
    if (raster_rounds < 1 || raster_rounds > 64)
        return fail(SM_ERR_INVALID_ARG, "raster rounds %d outside [1, 64]", raster_rounds);
    if (scatter_tiles < 1 || scatter_tiles > 4096)
        return fail(SM_ERR_INVALID_ARG, "scatter tiles %d outside [1, 4096]", scatter_tiles);
    m->use_queue = true;
    m->qB = frames_per_batch;
    m->qL = lookahead;
    m->qR = raster_rounds;
    m->qS = scatter_tiles;
    m->q_npix = (int64_t)H * W;
    return SM_OK;
}

sm_status sm_conf_features(sm_mesh *m, const void *d_probs, sm_dtype dtype, const float *d_scale,
                           const sm_intrinsics *d_K, const double *d_cam_to_world, int32_t N, int32_t H, int32_t W,
                           float *d_feat_out, int32_t *d_rows_out, void *stream)
{
    if (!m) return fail(SM_ERR_INVALID_ARG, "mesh is NULL");
    sm_status st = check_image(N, H, W);
    if (st != SM_OK) return st;
    if ((int)dtype < 0 || (int)dtype > 2) return fail(SM_ERR_INVALID_ARG, "unknown dtype %d", (int)dtype);
    if ((dtype == SM_F32) != (d_scale == nullptr) && N > 0) return fail(SM_ERR_INVALID_ARG, "scale given iff BF16/FP8");
    if (N == 0) return SM_OK;
    if (!d_probs || !d_K || !d_cam_to_world || !d_feat_out || !d_rows_out)
        return fail(SM_ERR_INVALID_ARG, "NULL pointer");
    DeviceGuard g(m->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t npix = (int64_t)H * W;
    const int B = batch_frames(m, npix, N);
    if ((st = prepare_frames(m, d_K, d_cam_to_world, N, npix, B, false, s)) != SM_OK) return st;
    const size_t esz = dtype_size(dtype);
    for (int f0 = 0; f0 < N; f0 += B) {
        const int nb = (N - f0 < B) ? N - f0 : B;
        if ((st = raster_only(m, f0, nb, H, W, m->keys, s)) != SM_OK) return st;
        lf::launch_conf_features(m->keys, npix * nb, H, W, m->verts, m->faces, m->F, d_K + f0,
                                 d_cam_to_world + 16 * (int64_t)f0,
                                 static_cast<const char *>(d_probs) + (size_t)f0 * npix * m->c * esz, dtype,
                                 d_scale ? d_scale + (size_t)f0 * npix : nullptr, m->c,
                                 d_feat_out + (size_t)f0 * npix * SM_CONF_FEATURES, s);
        LF_LAUNCHED("confidence features");
        // row map of the batch (re-arms the z-buffer)
        if ((st = resolve_only(m, f0, nb, H, W, m->keys, d_rows_out + (int64_t)f0 * npix, s, nullptr)) != SM_OK)
            return st;
    }
    return SM_OK;
}

sm_status sm_conf_weights(sm_mesh *m, const void *d_probs, sm_dtype dtype, const float *d_scale,
                          const sm_intrinsics *d_K, const double *d_cam_to_world, int32_t N, int32_t H, int32_t W,
                          const float *d_params, float *d_w_out, int32_t *d_rows_out, void *stream)
{
    if (!m) return fail(SM_ERR_INVALID_ARG, "mesh is NULL");
    sm_status st = check_image(N, H, W);
    if (st != SM_OK) return st;
    if ((int)dtype < 0 || (int)dtype > 2) return fail(SM_ERR_INVALID_ARG, "unknown dtype %d", (int)dtype);
    if ((dtype == SM_F32) != (d_scale == nullptr) && N > 0) return fail(SM_ERR_INVALID_ARG, "scale given iff BF16/FP8");
    if (N == 0) return SM_OK;
    if (!d_probs || !d_K || !d_cam_to_world || !d_params || !d_w_out || !d_rows_out)
        return fail(SM_ERR_INVALID_ARG, "NULL pointer");
    DeviceGuard g(m->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t npix = (int64_t)H * W;
    const int B = batch_frames(m, npix, N);
    if ((st = prepare_frames(m, d_K, d_cam_to_world, N, npix, B, false, s)) != SM_OK) return st;
    const size_t esz = dtype_size(dtype);
    for (int f0 = 0; f0 < N; f0 += B) {
        const int nb = (N - f0 < B) ? N - f0 : B;
        if ((st = raster_only(m, f0, nb, H, W, m->keys, s)) != SM_OK) return st;
        lf::launch_conf_weights(m->keys, npix * nb, H, W, m->verts, m->faces, m->F, d_K + f0,
                                d_cam_to_world + 16 * (int64_t)f0,
                                static_cast<const char *>(d_probs) + (size_t)f0 * npix * m->c * esz, dtype,
                                d_scale ? d_scale + (size_t)f0 * npix : nullptr, m->c, d_params,
                                d_w_out + (size_t)f0 * npix, m->texel_mode ? nullptr : d_rows_out + (int64_t)f0 * npix,
                                s);
        LF_LAUNCHED("confidence weights");
        // texel mode: the row of a pixel is its texel's (the resolve pass
        // writes it and re-arms the keys); face mode: the kernel wrote the
        // triangle and re-armed the keys itself
        if (m->texel_mode &&
            (st = resolve_only(m, f0, nb, H, W, m->keys, d_rows_out + (int64_t)f0 * npix, s)) != SM_OK)
            return st;
    }
    return SM_OK;
}

sm_status sm_conf_targets(sm_mesh *m, const void *d_probs, sm_dtype dtype, const float *d_scale,
                          const int32_t *d_rows, int64_t n_pixels, float *d_target_out, void *stream)
{
    if (!m) return fail(SM_ERR_INVALID_ARG, "mesh is NULL");
    if (!m->normalised) return fail(SM_ERR_STATE, "sm_conf_targets before sm_normalise");
    if (n_pixels < 0) return fail(SM_ERR_INVALID_ARG, "n_pixels < 0");
    if ((int)dtype < 0 || (int)dtype > 2) return fail(SM_ERR_INVALID_ARG, "unknown dtype %d", (int)dtype);
    if (n_pixels == 0) return SM_OK;
    if (!d_probs || !d_rows || !d_target_out || ((dtype != SM_F32) && !d_scale))
        return fail(SM_ERR_INVALID_ARG, "NULL pointer");
    DeviceGuard g(m->device);
    lf::launch_conf_targets(d_probs, dtype, d_scale, m->c, d_rows, n_pixels, m->labels8, m->n_x, d_target_out,
                            static_cast<cudaStream_t>(stream));
    LF_LAUNCHED("confidence targets");
    return SM_OK;
}

sm_status sm_conf_forward(const float *d_params, const float *d_feat, int64_t n, float *d_w_out, void *stream)
{
    if (n < 0) return fail(SM_ERR_INVALID_ARG, "n < 0");
    if (n == 0) return SM_OK;
    if (!d_params || !d_feat || !d_w_out) return fail(SM_ERR_INVALID_ARG, "NULL pointer");
    lf::launch_conf_forward(d_params, d_feat, n, d_w_out, static_cast<cudaStream_t>(stream));
    LF_LAUNCHED("confidence forward");
    return SM_OK;
}

sm_status sm_conf_train_step(float *d_params, const float *d_feat, const float *d_target, int64_t n, float lr,
                             float *d_grad_out, float *d_loss_out, void *stream)
{
    if (n < 0) return fail(SM_ERR_INVALID_ARG, "n < 0");
    if (!(lr >= 0.0f && lr < 1.0e6f)) return fail(SM_ERR_INVALID_ARG, "learning rate %g", (double)lr);
    if (!d_params || !d_grad_out || !d_loss_out || (n > 0 && (!d_feat || !d_target)))
        return fail(SM_ERR_INVALID_ARG, "NULL pointer");
    const cudaError_t e = lf::launch_conf_train_step(d_params, d_feat, d_target, n, lr, d_grad_out, d_loss_out,
                                                     static_cast<cudaStream_t>(stream));
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return fail(SM_ERR_OOM, "confidence training step: stream-ordered allocation of its sums");
    }
    if (e != cudaSuccess) return cuda_fail(e, "confidence training step");
    return SM_OK;
}

sm_status sm_conf_train_step_indexed(float *d_params, const float *d_feat, const float *d_target, int64_t n_obs,
                                     const int64_t *d_idx, int64_t m, float lr, float *d_grad_out, float *d_loss_out,
                                     void *stream)
{
    if (m < 0 || n_obs < 0) return fail(SM_ERR_INVALID_ARG, "m < 0 or n_obs < 0");
    if (m > 0 && n_obs == 0) return fail(SM_ERR_INVALID_ARG, "indices into an empty set of observations");
    if (!(lr >= 0.0f && lr < 1.0e6f)) return fail(SM_ERR_INVALID_ARG, "learning rate %g", (double)lr);
    if (!d_params || !d_grad_out || !d_loss_out || (m > 0 && (!d_feat || !d_target || !d_idx)))
        return fail(SM_ERR_INVALID_ARG, "NULL pointer");
    const cudaError_t e = lf::launch_conf_train_step(d_params, d_feat, d_target, m, lr, d_grad_out, d_loss_out,
                                                     static_cast<cudaStream_t>(stream), d_idx, n_obs);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return fail(SM_ERR_OOM, "confidence training step: stream-ordered allocation of its sums");
    }
    if (e != cudaSuccess) return cuda_fail(e, "confidence training step");
    return SM_OK;
}

sm_status sm_host_alloc(uint64_t bytes, void **out)
{
    if (!out || bytes == 0) return fail(SM_ERR_INVALID_ARG, "sm_host_alloc: NULL out or zero bytes");
    *out = nullptr;
    const cudaError_t e = cudaHostAlloc(out, (size_t)bytes, cudaHostAllocDefault);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *out = nullptr;
        return fail(SM_ERR_OOM, "cudaHostAlloc(%llu bytes): %s", (unsigned long long)bytes, cudaGetErrorString(e));
    }
    return SM_OK;
}

sm_status sm_host_free(void *p)
{
    if (!p) return SM_OK;
    const cudaError_t e = cudaFreeHost(p);
    return e == cudaSuccess ? SM_OK : cuda_fail(e, "cudaFreeHost");
}

namespace {
// Blocks of sm_device_alloc: compressible mappings need their size and handle
// to be released, plain blocks only their device.
struct DeviceBlock {
    int device;
    sm_mesh::VmmBlock vmm;
};
std::mutex g_blocks_mu;
std::unordered_map<void *, DeviceBlock> g_blocks;
}  // namespace

sm_status sm_device_alloc(int32_t device, uint64_t bytes, int32_t flags, void **out, int32_t *compressed_out)
{
    if (compressed_out) *compressed_out = 0;
    if (out) *out = nullptr;
    if (!out || bytes == 0) return fail(SM_ERR_INVALID_ARG, "sm_device_alloc: NULL out or zero bytes");
    if (flags & ~SM_DEVICE_COMPRESSIBLE) return fail(SM_ERR_INVALID_ARG, "sm_device_alloc: unknown flags 0x%x", flags);
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess) {
        cudaGetLastError();
        ndev = 0;
    }
    if (device < 0 || device >= ndev) return fail(SM_ERR_INVALID_ARG, "sm_device_alloc: no device %d", device);
    DeviceGuard g(device);
    DeviceBlock blk{device, {}};
    void *p = nullptr;
    size_t mapped = 0;
    unsigned long long h = 0;
    if ((flags & SM_DEVICE_COMPRESSIBLE) && compressible_alloc(device, (size_t)bytes, &p, &mapped, &h)) {
        blk.vmm = sm_mesh::VmmBlock{p, mapped, h};
        if (compressed_out) *compressed_out = 1;
    } else {
        const cudaError_t e = device_alloc(&p, (size_t)bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return cuda_fail(e, "sm_device_alloc");
        }
    }
    {
        std::lock_guard<std::mutex> lk(g_blocks_mu);
        g_blocks[p] = blk;
    }
    *out = p;
    return SM_OK;
}

sm_status sm_device_free(void *p)
{
    if (!p) return SM_OK;
    DeviceBlock blk;
    {
        std::lock_guard<std::mutex> lk(g_blocks_mu);
        auto it = g_blocks.find(p);
        if (it == g_blocks.end()) return fail(SM_ERR_INVALID_ARG, "sm_device_free: not a block of sm_device_alloc");
        blk = it->second;
        g_blocks.erase(it);
    }
    DeviceGuard g(blk.device);
    if (!blk.vmm.p) {
        const cudaError_t e = cudaFree(p);
        return e == cudaSuccess ? SM_OK : cuda_fail(e, "sm_device_free");
    }
    // a mapping is released only once no work on the device can still use it
    const cudaError_t e = cudaDeviceSynchronize();
    compressible_free(blk.vmm.p, blk.vmm.mapped, blk.vmm.handle);
    return e == cudaSuccess ? SM_OK : cuda_fail(e, "sm_device_free");
}

sm_status sm_fuse_render_host(sm_mesh *m, const void *h_probs, sm_dtype dtype, const float *h_scale,
                              const sm_intrinsics *h_K, const double *h_cam_to_world, int32_t N, int32_t H, int32_t W,
                              uint8_t *h_labels_out, void *stream)
{
    if (!m) return fail(SM_ERR_INVALID_ARG, "mesh is NULL");
    sm_status st = check_image(N, H, W);
    if (st != SM_OK) return st;
    if ((int)dtype < 0 || (int)dtype > 2) return fail(SM_ERR_INVALID_ARG, "unknown dtype %d", (int)dtype);
    if (dtype == SM_F32 && h_scale) return fail(SM_ERR_INVALID_ARG, "F32 probabilities take no scale");
    if (dtype != SM_F32 && !h_scale && N > 0) return fail(SM_ERR_INVALID_ARG, "BF16/FP8 need a per-pixel scale");
    if (N == 0) return SM_OK;
    if (!h_probs || !h_K || !h_cam_to_world || !h_labels_out) return fail(SM_ERR_INVALID_ARG, "NULL host pointer");
    DeviceGuard g(m->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    constexpr int NC = sm_mesh::kCopyStreams;
    const int64_t npix = (int64_t)H * W;
    const int B = batch_frames(m, npix, N, false);  // small batches keep copies and fusion overlapped
    const size_t frame_bytes = (size_t)npix * m->c * dtype_size(dtype);
    const size_t probs_slot = ((size_t)B * frame_bytes + 255) & ~(size_t)255;
    const size_t slot_bytes = probs_slot + (dtype != SM_F32 ? (((size_t)B * npix * 4 + 255) & ~(size_t)255) : 0);
    if ((st = grow(&m->hstage, &m->hstage_cap, 2 * (int64_t)slot_bytes, s, -1, "host staging")) != SM_OK) return st;
    if ((st = grow_compressible(m, &m->hids, &m->hids_cap, &m->hids_blk, (int64_t)N * npix, s, -1, "row maps")) !=
        SM_OK)
        return st;
    if ((st = grow_compressible(m, &m->hlabels, &m->hlabels_cap, &m->hlabels_blk, (int64_t)N * npix, s, -1,
                                "label images")) != SM_OK)
        return st;
    if ((st = grow(&m->hcam, &m->hcam_cap, 20 * (int64_t)N, s, -1, "cameras")) != SM_OK) return st;
    sm_intrinsics *d_K = reinterpret_cast<sm_intrinsics *>(m->hcam);
    double *d_T = m->hcam + 4 * (int64_t)N;
    LF_CUDA(cudaMemcpyAsync(d_K, h_K, sizeof(sm_intrinsics) * N, cudaMemcpyHostToDevice, s), "copy cameras");
    LF_CUDA(cudaMemcpyAsync(d_T, h_cam_to_world, sizeof(double) * 16 * N, cudaMemcpyHostToDevice, s), "copy cameras");
    // the copy stream may refill a staging slot once the fusion reading it is done
    LF_CUDA(cudaEventRecord(m->ev_free[0], s), "event");
    LF_CUDA(cudaEventRecord(m->ev_free[1], s), "event");
    for (int b = 0, f0 = 0; f0 < N; ++b, f0 += B) {
        const int nb = (N - f0 < B) ? N - f0 : B;
        const int slot = b & 1;
        uint8_t *dp = m->hstage + slot * slot_bytes;
        float *dsc = dtype != SM_F32 ? reinterpret_cast<float *>(dp + probs_slot) : nullptr;
        // the batch's predictions in NC parts of whole 4 KiB pages, one per copy stream
        const size_t total = (size_t)nb * frame_bytes;
        const size_t part = ((total + NC - 1) / NC + 4095) & ~(size_t)4095;
        const uint8_t *src = static_cast<const uint8_t *>(h_probs) + (size_t)f0 * frame_bytes;
        for (int k = 0; k < NC; ++k) {
            cudaStream_t cs = m->cstream[k];
            LF_CUDA(cudaStreamWaitEvent(cs, m->ev_free[slot], 0), "event");
            const size_t off = (size_t)k * part;
            if (off < total)
                LF_CUDA(cudaMemcpyAsync(dp + off, src + off, total - off < part ? total - off : part,
                                        cudaMemcpyHostToDevice, cs),
                        "copy predictions");
            if (dsc && k == NC - 1)
                LF_CUDA(cudaMemcpyAsync(dsc, h_scale + (size_t)f0 * npix, (size_t)nb * npix * sizeof(float),
                                        cudaMemcpyHostToDevice, cs),
                        "copy scales");
            LF_CUDA(cudaEventRecord(m->ev_h2d[slot][k], cs), "event");
            LF_CUDA(cudaStreamWaitEvent(s, m->ev_h2d[slot][k], 0), "event");
        }
        if ((st = sm_fuse_frames(m, dp, dtype, dsc, d_K + f0, d_T + 16 * (int64_t)f0, nb, H, W,
                                 m->hids + (int64_t)f0 * npix, stream)) != SM_OK)
            return st;
        LF_CUDA(cudaEventRecord(m->ev_free[slot], s), "event");
    }
    if ((st = sm_normalise(m, nullptr, nullptr, stream)) != SM_OK) return st;
    if ((st = sm_render_idmap(m, m->hids, (int64_t)N * npix, m->hlabels, stream)) != SM_OK) return st;
    LF_CUDA(cudaMemcpyAsync(h_labels_out, m->hlabels, (size_t)N * npix, cudaMemcpyDeviceToHost, s), "copy labels");
    LF_CUDA(cudaStreamSynchronize(s), "synchronise");
    return SM_OK;
}

sm_status sm_reset(sm_mesh *m, void *stream)
{
    if (!m) return fail(SM_ERR_INVALID_ARG, "mesh is NULL");
    DeviceGuard g(m->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t rows = m->n_x > 0 ? m->n_x : 1;
    LF_CUDA(cudaMemsetAsync(m->acc, 0, (size_t)rows * m->c * sizeof(float), s), "reset");
    LF_CUDA(cudaMemsetAsync(m->cnt, 0, (size_t)rows * sizeof(uint32_t), s), "reset");
    m->normalised = false;
    return SM_OK;
}

sm_status sm_read_state(sm_mesh *m, float *d_acc_out, uint32_t *d_cnt_out, void *stream)
{
    if (!m) return fail(SM_ERR_INVALID_ARG, "mesh is NULL");
    DeviceGuard g(m->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (d_acc_out && m->n_x > 0)
        LF_CUDA(cudaMemcpyAsync(d_acc_out, m->acc, (size_t)m->n_x * m->c * sizeof(float), cudaMemcpyDeviceToDevice,
                                s),
                "read state");
    if (d_cnt_out && m->n_x > 0)
        LF_CUDA(cudaMemcpyAsync(d_cnt_out, m->cnt, (size_t)m->n_x * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s),
                "read state");
    return SM_OK;
}

sm_status sm_load_state(sm_mesh *m, const float *d_acc, const uint32_t *d_cnt, void *stream)
{
    if (!m) return fail(SM_ERR_INVALID_ARG, "mesh is NULL");
    if (m->n_x > 0 && (!d_acc || !d_cnt)) return fail(SM_ERR_INVALID_ARG, "NULL state pointer");
    DeviceGuard g(m->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (m->n_x > 0) {
        LF_CUDA(cudaMemcpyAsync(m->acc, d_acc, (size_t)m->n_x * m->c * sizeof(float), cudaMemcpyDeviceToDevice, s),
                "load state");
        LF_CUDA(cudaMemcpyAsync(m->cnt, d_cnt, (size_t)m->n_x * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s),
                "load state");
    }
    m->normalised = false;
    return SM_OK;
}

sm_status sm_check(sm_mesh *m, void *stream)
{
    if (!m) return fail(SM_ERR_INVALID_ARG, "mesh is NULL");
    DeviceGuard g(m->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int32_t latched = 0;
    LF_CUDA(cudaMemcpyAsync(&latched, m->err, sizeof(int32_t), cudaMemcpyDeviceToHost, s), "read error latch");
    LF_CUDA(cudaStreamSynchronize(s), "synchronise");
    if (latched != lf::kErrNone) {
        LF_CUDA(cudaMemsetAsync(m->err, 0, sizeof(int32_t), s), "clear error latch");
        LF_CUDA(cudaStreamSynchronize(s), "synchronise");
        if (latched == lf::kErrTimeout) {
            // the kernel that gave up left part of its scratch as it was:
            // re-arm the z-buffers and clear the row histograms so that the
            // next call starts clean (the accumulators are the caller's to
            // reset)
            if (m->keys) LF_CUDA(cudaMemsetAsync(m->keys, 0xFF, (size_t)m->keys_cap * sizeof(*m->keys), s), "re-arm");
            if (m->fcnt) LF_CUDA(cudaMemsetAsync(m->fcnt, 0, (size_t)m->fcnt_cap * sizeof(*m->fcnt), s), "re-arm");
            LF_CUDA(cudaStreamSynchronize(s), "synchronise");
            return fail(SM_ERR_TIMEOUT, "a bounded wait inside a kernel gave up (code %d)", latched);
        }
        const char *what = latched == lf::kErrFaceIndex   ? "a face references a vertex outside [0, V)"
                           : latched == lf::kErrRowRange  ? "a row index outside [0, n_x) reached the scatter"
                           : latched == lf::kErrTexelRes  ? "texel steps out of range"
                                                          : "internal error";
        return fail(SM_ERR_INTERNAL, "%s (code %d)", what, latched);
    }
    return SM_OK;
}

int64_t sm_num_rows(const sm_mesh *m) { return m ? m->n_x : -1; }

int32_t sm_num_classes(const sm_mesh *m) { return m ? m->c : -1; }

sm_status sm_mesh_free(sm_mesh *m)
{
    if (!m) return SM_OK;
    {
        DeviceGuard g(m->device);
        cudaDeviceSynchronize();
        void *bufs[] = {m->verts, m->faces, m->row0, m->texinfo, m->acc, m->cnt, m->labels8, m->err, m->cams,
                        m->keys_blk.p ? nullptr : m->keys, m->idbuf_blk.p ? nullptr : m->idbuf, m->wbuf,
                        m->fcnt_blk.p ? nullptr : m->fcnt, m->bounds, m->hstage,
                        m->hids_blk.p ? nullptr : m->hids, m->hlabels_blk.p ? nullptr : m->hlabels, m->hcam,
                        m->clist, m->ccount, m->area, m->qctr};
        for (void *b : bufs)
            if (b) cudaFree(b);
        for (const sm_mesh::VmmBlock &b : {m->keys_blk, m->idbuf_blk, m->fcnt_blk, m->hids_blk, m->hlabels_blk})
            if (b.p) compressible_free(b.p, b.mapped, b.handle);
        for (const auto &r : m->retired) compressible_free(r.p, r.mapped, r.handle);
        if (m->rstream) cudaStreamDestroy(m->rstream);
        for (cudaStream_t cs : m->cstream)
            if (cs) cudaStreamDestroy(cs);
        cudaEvent_t evs[] = {m->ev_start,  m->ev_rast[0], m->ev_rast[1], m->ev_scat[0],
                             m->ev_scat[1], m->ev_free[0], m->ev_free[1]};
        for (cudaEvent_t e : evs)
            if (e) cudaEventDestroy(e);
        for (auto &slot : m->ev_h2d)
            for (cudaEvent_t e : slot)
                if (e) cudaEventDestroy(e);
        for (int k = 0; k < SM_K_COUNT_KINDS; ++k)
            for (auto &p : m->ev[k]) {
                cudaEventDestroy(p.a);
                cudaEventDestroy(p.b);
            }
    }
    delete m;
    return SM_OK;
}

sm_status sm_render_rows_noalloc(const float *d_vertices, int64_t V, const int32_t *d_faces, int64_t F,
                                 const sm_intrinsics *d_K, const double *d_cam_to_world, int32_t N, int32_t H,
                                 int32_t W, int32_t *d_idmap_out, void *stream)
{
    sm_status st = check_image(N, H, W);
    if (st != SM_OK) return st;
    if (V < 0 || F < 0 || V >= (1LL << 31) || F >= (1LL << 31))
        return fail(SM_ERR_INVALID_ARG, "V or F outside [0, 2^31)");
    if ((int64_t)H * W > SM_NOALLOC_MAX_PIXELS)
        return fail(SM_ERR_INVALID_ARG, "H x W = %lld pixels exceeds the static scratch (%d)", (long long)H * W,
                    SM_NOALLOC_MAX_PIXELS);
    if (N > SM_NOALLOC_MAX_FRAMES)
        return fail(SM_ERR_INVALID_ARG, "N = %d frames exceeds the static scratch (%d)", N, SM_NOALLOC_MAX_FRAMES);
    if (N == 0) return SM_OK;
    if (!d_K || !d_cam_to_world || !d_idmap_out || (F > 0 && (!d_vertices || !d_faces)))
        return fail(SM_ERR_INVALID_ARG, "NULL pointer");
    // the call runs on the device that holds the output; every input must be
    // device memory of that same device (or memory it can address directly)
    int dev = -1;
    {
        cudaPointerAttributes at{};
        if (cudaPointerGetAttributes(&at, d_idmap_out) != cudaSuccess || at.type != cudaMemoryTypeDevice) {
            cudaGetLastError();
            return fail(SM_ERR_INVALID_ARG, "d_idmap_out is not device memory");
        }
        dev = at.device;
        const void *ins[] = {d_K, d_cam_to_world, F > 0 ? d_vertices : nullptr, F > 0 ? d_faces : nullptr};
        const char *names[] = {"d_K", "d_cam_to_world", "d_vertices", "d_faces"};
        for (int k = 0; k < 4; ++k) {
            if (!ins[k]) continue;
            cudaPointerAttributes ai{};
            if (cudaPointerGetAttributes(&ai, ins[k]) != cudaSuccess) {
                cudaGetLastError();
                return fail(SM_ERR_INVALID_ARG, "%s: unknown pointer", names[k]);
            }
            const bool same_device = ai.type == cudaMemoryTypeDevice && ai.device == dev;
            const bool addressable = ai.type == cudaMemoryTypeManaged || (ai.type == cudaMemoryTypeHost && ai.devicePointer);
            if (!same_device && !addressable)
                return fail(SM_ERR_INVALID_ARG, "%s is not memory of device %d, which holds d_idmap_out", names[k], dev);
        }
    }
    DeviceGuard g(dev);
    cudaError_t e = lf::launch_render_rows_noalloc(d_vertices, V, d_faces, F, d_K, d_cam_to_world, N, H, W,
                                                   d_idmap_out, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "render rows (no allocation)");
    return SM_OK;
}

sm_status sm_profile_enable(sm_mesh *m, int32_t on)
{
    if (!m) return fail(SM_ERR_INVALID_ARG, "mesh is NULL");
    m->prof = on != 0;
    return SM_OK;
}

sm_status sm_profile_read(sm_mesh *m, sm_kernel kernel, int64_t *launches, double *total_ms)
{
    if (!m) return fail(SM_ERR_INVALID_ARG, "mesh is NULL");
    if ((int)kernel < 0 || (int)kernel >= SM_K_COUNT_KINDS) return fail(SM_ERR_INVALID_ARG, "unknown kernel");
    DeviceGuard g(m->device);
    const int k = (int)kernel;
    double tot = 0.0;
    for (size_t i = 0; i < m->ev_used[k]; ++i) {
        LF_CUDA(cudaEventSynchronize(m->ev[k][i].b), "profile");
        float ms = 0.0f;
        LF_CUDA(cudaEventElapsedTime(&ms, m->ev[k][i].a, m->ev[k][i].b), "profile");
        tot += ms;
    }
    if (launches) *launches = m->ev_kernels[k];
    if (total_ms) *total_ms = tot;
    m->ev_used[k] = 0;
    m->ev_kernels[k] = 0;
    return SM_OK;
}

}  // extern "C"
