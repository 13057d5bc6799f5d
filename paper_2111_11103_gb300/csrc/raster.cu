// Renderer kernels (Sec. 3.3.1): per-frame camera set-up, triangle raster with
// a 64-bit z-buffer key, and the resolve of the z-buffer into row indices
// l = id_t + id_x (Eq. texel-in-array).
//
// Determinism: every floating-point step uses explicit round-to-nearest
// intrinsics (__fmul_rn, __fadd_rn, __fdiv_rn, __dmul_rn, __dadd_rn), which the
// compiler never contracts into FMAs, so the integer decisions (snapped vertex
// positions, coverage, the depth key) are the same on every run and match the
// project's raster reading bit for bit.
#include "lf_internal.cuh"
#include "ptx.cuh"
#include "raster_dev.cuh"

namespace lf {
namespace {

// Camera set-up in binary64 (the only binary64 work on the device): world to
// camera R = Rcw^T, t = -R C; image rows scaled by 256 (exact) for the
// 1/256-pixel snap grid; each entry rounded to binary32 once.
__global__ void k_project(const sm_intrinsics *__restrict__ Ks, const double *__restrict__ Ts, int N,
                          Camera *__restrict__ out)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double *T = Ts + 16 * (int64_t)i;
    const sm_intrinsics K = Ks[i];
    double R[3][3], C[3], t[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
#pragma unroll
        for (int c = 0; c < 3; ++c) R[r][c] = T[c * 4 + r];
        C[r] = T[r * 4 + 3];
    }
#pragma unroll
    for (int r = 0; r < 3; ++r)
        t[r] = -__dadd_rn(__dadd_rn(__dmul_rn(R[r][0], C[0]), __dmul_rn(R[r][1], C[1])), __dmul_rn(R[r][2], C[2]));
    Camera cam;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        cam.a[c] = __double2float_rn(__dmul_rn(256.0, __dadd_rn(__dmul_rn(K.fx, R[0][c]), __dmul_rn(K.cx, R[2][c]))));
        cam.a[4 + c] =
            __double2float_rn(__dmul_rn(256.0, __dadd_rn(__dmul_rn(K.fy, R[1][c]), __dmul_rn(K.cy, R[2][c]))));
        cam.a[8 + c] = __double2float_rn(R[2][c]);
    }
    cam.a[3] = __double2float_rn(__dmul_rn(256.0, __dadd_rn(__dmul_rn(K.fx, t[0]), __dmul_rn(K.cx, t[2]))));
    cam.a[7] = __double2float_rn(__dmul_rn(256.0, __dadd_rn(__dmul_rn(K.fy, t[1]), __dmul_rn(K.cy, t[2]))));
    cam.a[11] = __double2float_rn(t[2]);
    out[i] = cam;
}

// World-space bounding box of every cluster of 32 consecutive faces (one warp
// per cluster); clusters without a valid face are marked with min.w = 1.
__global__ void k_cluster_bounds(const float4 *__restrict__ V, const int4 *__restrict__ faces, int64_t F,
                                 float4 *__restrict__ bounds)
{
    const int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t cl = f / kClusterFaces;
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    bool any = false;
    if (f < F) {
        const int4 fc = faces[f];
        if (fc.w) {
            any = true;
            const float4 p[3] = {V[fc.x], V[fc.y], V[fc.z]};
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                lo[0] = fminf(lo[0], p[k].x);
                lo[1] = fminf(lo[1], p[k].y);
                lo[2] = fminf(lo[2], p[k].z);
                hi[0] = fmaxf(hi[0], p[k].x);
                hi[1] = fmaxf(hi[1], p[k].y);
                hi[2] = fmaxf(hi[2], p[k].z);
            }
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            lo[d] = fminf(lo[d], __shfl_xor_sync(0xffffffffu, lo[d], off));
            hi[d] = fmaxf(hi[d], __shfl_xor_sync(0xffffffffu, hi[d], off));
        }
    }
    any = __any_sync(0xffffffffu, any);
    if ((threadIdx.x & 31) == 0 && cl * kClusterFaces < F) {
        bounds[2 * cl] = make_float4(lo[0], lo[1], lo[2], any ? 0.0f : 1.0f);
        bounds[2 * cl + 1] = make_float4(hi[0], hi[1], hi[2], 0.0f);
    }
}

// Cluster cull of one batch: one thread per (cluster, frame) applies the
// conservative frustum test (cluster_may_be_visible) and appends the clusters
// that may be visible to its frame's list (one atomic per warp).
// blockIdx.y = frame in the batch.
__global__ void __launch_bounds__(256) k_cull_clusters(const float4 *__restrict__ bounds, int64_t ncl,
                                                       const Camera *__restrict__ cams, int frame0, int H, int W,
                                                       int32_t *__restrict__ list, uint32_t *__restrict__ count)
{
    __shared__ float A[12];
    const int b = blockIdx.y;
    if (threadIdx.x < 12) A[threadIdx.x] = cams[frame0 + b].a[threadIdx.x];
    __syncthreads();
    const int64_t cl = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool keep = cl < ncl && cluster_may_be_visible(bounds, cl, A, H, W);
    const unsigned mask = __ballot_sync(0xffffffffu, keep);
    if (!mask) return;
    const int lane = threadIdx.x & 31;
    uint32_t base = 0;
    if (lane == __ffs(mask) - 1) base = atomicAdd(count + b, (uint32_t)__popc(mask));
    base = __shfl_sync(0xffffffffu, base, __ffs(mask) - 1);
    if (keep) list[(int64_t)b * ncl + base + __popc(mask & ((1u << lane) - 1u))] = (int32_t)cl;
}

// Raster of the listed clusters: one warp per cluster and one thread per
// face; blockIdx.y = frame in the batch, the x blocks' warps stride over the
// frame's list.  Set-up and box walk as in raster_face.
__global__ void __launch_bounds__(256, 4) k_raster_list(const float4 *__restrict__ V, const int4 *__restrict__ faces,
                                                     int64_t F, int64_t ncl, const int32_t *__restrict__ list,
                                                     const uint32_t *__restrict__ count,
                                                     const Camera *__restrict__ cams, int frame0, int H, int W,
                                                     unsigned long long *__restrict__ keys)
{
    __shared__ float A[12];
    const int b = blockIdx.y;
    if (threadIdx.x < 12) A[threadIdx.x] = cams[frame0 + b].a[threadIdx.x];
    __syncthreads();
    const uint32_t n = count[b];
    const int warps = blockDim.x >> 5;
    unsigned long long *frame_keys = keys + (int64_t)b * H * W;
    for (uint32_t j = blockIdx.x * warps + (threadIdx.x >> 5); j < n; j += gridDim.x * warps) {
        const int64_t cl = list[(int64_t)b * ncl + j];
        raster_face(A, V, faces, F, cl * kClusterFaces + (threadIdx.x & 31), H, W, frame_keys);
    }
}

// z-buffer -> row map, and re-arms the z-buffer for the next batch.  For a
// subdivided triangle (s > 1) the winning triangle's perspective-correct
// barycentrics are recomputed with the same operations as the raster:
// beta_k = (float)E_k * iz_k / ((w0 + w1) + w2); u, v are the barycentrics of
// the vertices after the uv origin; the texel cell (i, j) is
// (floor(s u), floor(s v)) clamped into the triangle and id_x = T(i + j) + j.
// Row of pixel p of the batch whose nearest surface is triangle f, in texel
// mode (called per pixel, kept out of line so that the resolve loop stays
// small).
__device__ __noinline__ int32_t texel_row(int f, int64_t p, int H, int W, const int32_t *__restrict__ row0,
                                          const int32_t *__restrict__ texinfo, const float4 *__restrict__ V,
                                          const int4 *__restrict__ faces, const Camera *__restrict__ cams, int frame0)
{
    const int info = texinfo[f];
    const int s = info & 0xFFFF;
    const int o = info >> 16;
    int idx = 0;
    if (s > 1) {
        const int64_t npix = (int64_t)H * W;
        const int b = (int)frame_of(p, npix);
        const int64_t q = p - (int64_t)b * npix;
        const int py = (int)(q / W), px = (int)(q - (int64_t)py * W);
        const float *A = cams[frame0 + b].a;
        Tri t;
        setup_triangle(A, V, faces[f], t);
        float w[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) w[k] = fmul(i2f(edge_at(t, k, 256LL * px, 256LL * py)), t.iz[k]);
        const float num = fadd(fadd(w[0], w[1]), w[2]);
        float beta[3];
        beta[0] = fdiv(w[0], num);
        beta[t.swapped ? 2 : 1] = fdiv(w[1], num);
        beta[t.swapped ? 1 : 2] = fdiv(w[2], num);
        const float u = beta[(o + 1) % 3], v = beta[(o + 2) % 3];
        const float fs = (float)s;
        int i = (int)floorf(fmul(fs, u));
        i = min(max(i, 0), s - 1);
        int j = (int)floorf(fmul(fs, v));
        j = min(max(j, 0), s - 1 - i);
        idx = (i + j) * (i + j + 1) / 2 + j;
    }
    return row0[f] + idx;
}

// kPixUnroll pixels per thread (see kPixThreads): the keys are loaded first,
// then resolved; keys left empty by the raster are not written again.
template <bool TEXEL>
__global__ void __launch_bounds__(kPixThreads) k_resolve(unsigned long long *__restrict__ keys, int64_t total, int H,
                                                         int W, const int32_t *__restrict__ row0,
                                                         const int32_t *__restrict__ texinfo,
                                                         const float4 *__restrict__ V, const int4 *__restrict__ faces,
                                                         const Camera *__restrict__ cams, int frame0,
                                                         int32_t *__restrict__ idmap, int32_t *__restrict__ idmap2)
{
    const int64_t base = (int64_t)blockIdx.x * kPixPerBlock;
    unsigned long long key[kPixUnroll];
#pragma unroll
    for (int j = 0; j < kPixUnroll; ++j) {
        const int64_t p = base + j * kPixThreads + threadIdx.x;
        key[j] = p < total ? keys[p] : kEmptyKey;
    }
#pragma unroll
    for (int j = 0; j < kPixUnroll; ++j) {
        const int64_t p = base + j * kPixThreads + threadIdx.x;
        if (p < total) {
            int32_t row = -1;
            if (key[j] != kEmptyKey) {
                keys[p] = kEmptyKey;
                const int f = (int)(unsigned int)key[j];
                row = TEXEL ? texel_row(f, p, H, W, row0, texinfo, V, faces, cams, frame0) : f;
            }
            idmap[p] = row;
            if (idmap2) idmap2[p] = row;
        }
    }
}

// ---- raster for the allocation-free entry point (sm_render_rows_noalloc) ----

// Same coverage and depth rules as k_raster, for one frame, reading the
// caller's plain V x 3 vertices and F x 3 indices directly (no packed copies,
// no cluster culling).  Faces with an index outside [0, V) are never drawn.
__global__ void __launch_bounds__(256) k_raster_flat(const float *__restrict__ V, int64_t nV,
                                                     const int32_t *__restrict__ faces, int64_t F,
                                                     const Camera *__restrict__ cam, int H, int W,
                                                     unsigned long long *__restrict__ keys)
{
    __shared__ float A[12];
    if (threadIdx.x < 12) A[threadIdx.x] = cam->a[threadIdx.x];
    __syncthreads();
    const int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= F) return;
    const int i0 = faces[3 * f], i1 = faces[3 * f + 1], i2 = faces[3 * f + 2];
    if (i0 < 0 || i0 >= nV || i1 < 0 || i1 >= nV || i2 < 0 || i2 >= nV) return;
    float4 P[3];
    const int ix[3] = {i0, i1, i2};
#pragma unroll
    for (int k = 0; k < 3; ++k) P[k] = make_float4(V[3 * (int64_t)ix[k]], V[3 * (int64_t)ix[k] + 1],
                                                   V[3 * (int64_t)ix[k] + 2], 0.0f);
    Tri t;
    if (!setup_triangle(A, P, make_int4(0, 1, 2, 1), t, H, W)) return;
    int minx = min(t.x[0], min(t.x[1], t.x[2])), maxx = max(t.x[0], max(t.x[1], t.x[2]));
    int miny = min(t.y[0], min(t.y[1], t.y[2])), maxy = max(t.y[0], max(t.y[1], t.y[2]));
    int x0 = max(ceil256(minx), 0), x1 = min(floor256(maxx), W - 1);
    int y0 = max(ceil256(miny), 0), y1 = min(floor256(maxy), H - 1);
    if (x0 > x1 || y0 > y1) return;
    if (maxx - minx <= (1 << 14) && maxy - miny <= (1 << 14))
        raster_box<int>(t, x0, x1, y0, y1, (unsigned int)f, keys, W);
    else
        raster_box<long long>(t, x0, x1, y0, y1, (unsigned int)f, keys, W);
}

__global__ void k_fill_empty(unsigned long long *__restrict__ keys, int64_t n)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) keys[i] = kEmptyKey;
}

}  // namespace

// Scratch of sm_render_rows_noalloc, in the library's static device memory
// (present on every GPU that loads the library, for the life of the process):
// the z-buffer of one frame (SM_NOALLOC_MAX_PIXELS 64-bit keys) followed by
// the per-frame cameras (SM_NOALLOC_MAX_FRAMES x 48 bytes = 6 words each).
// Host code may not use this name as an address; it asks the runtime for the
// device address of the current device's copy (below).
static __device__ __align__(256) unsigned long long
    g_noalloc_scratch[SM_NOALLOC_MAX_PIXELS + 6 * SM_NOALLOC_MAX_FRAMES];

// Device address of the static scratch on the current device.  Looked up on
// every call (cudaGetSymbolAddress needs that device current, allocates
// nothing and is cheap), so that no address outlives the context it belongs
// to (after a device reset the module, and with it the array, is reloaded).
cudaError_t noalloc_scratch(unsigned long long **out)
{
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    *out = static_cast<unsigned long long *>(p);
    return cudaSuccess;
}

// Renders N frames into d_idmap_out with the static scratch (see labelfuse.h).
cudaError_t launch_render_rows_noalloc(const float *V, int64_t nV, const int32_t *faces, int64_t F,
                                       const sm_intrinsics *K, const double *T, int N, int H, int W, int32_t *idmap,
                                       cudaStream_t s)
{
    unsigned long long *scratch = nullptr;
    cudaError_t e = noalloc_scratch(&scratch);
    if (e != cudaSuccess) return e;
    unsigned long long *keys = scratch;
    Camera *cams = reinterpret_cast<Camera *>(scratch + SM_NOALLOC_MAX_PIXELS);
    const int64_t npix = (int64_t)H * W;
    // the scratch keeps the previous call's contents: re-arm the z-buffer
    k_fill_empty<<<(unsigned)((npix + 255) / 256), 256, 0, s>>>(keys, npix);
    k_project<<<(N + 127) / 128, 128, 0, s>>>(K, T, N, cams);
    for (int i = 0; i < N; ++i) {
        if (F > 0) k_raster_flat<<<(unsigned)((F + 255) / 256), 256, 0, s>>>(V, nV, faces, F, cams + i, H, W, keys);
        // resolve in face mode (row = triangle); re-arms the z-buffer
        k_resolve<false><<<(unsigned)((npix + kPixPerBlock - 1) / kPixPerBlock), kPixThreads, 0, s>>>(
            keys, npix, H, W, nullptr, nullptr, nullptr, nullptr, cams, i, idmap + (int64_t)i * npix, nullptr);
    }
    return cudaGetLastError();
}

void launch_project(const sm_intrinsics *K, const double *T, int N, Camera *out, cudaStream_t s)
{
    if (N <= 0) return;
    k_project<<<(N + 127) / 128, 128, 0, s>>>(K, T, N, out);
}

void launch_cluster_bounds(const float4 *V, const int4 *faces, int64_t F, float4 *bounds, cudaStream_t s)
{
    if (F <= 0) return;
    k_cluster_bounds<<<(unsigned)((F + 255) / 256), 256, 0, s>>>(V, faces, F, bounds);
}

void launch_raster(const float4 *V, const int4 *faces, int64_t F, const float4 *bounds, const Camera *cams,
                   int frame0, int nb, int H, int W, unsigned long long *keys, int32_t *list, uint32_t *count,
                   cudaStream_t s)
{
    if (F <= 0 || nb <= 0) return;
    const int64_t ncl = (F + kClusterFaces - 1) / kClusterFaces;
    cudaMemsetAsync(count, 0, (size_t)nb * sizeof(uint32_t), s);
    k_cull_clusters<<<dim3((unsigned)((ncl + 255) / 256), (unsigned)nb), 256, 0, s>>>(bounds, ncl, cams, frame0, H,
                                                                                     W, list, count);
    // enough warps per frame for a typical visible fraction; warps loop over longer lists
    const int64_t bx = ncl / 32 < 1 ? 1 : (ncl / 32 > 128 ? 128 : ncl / 32);
    k_raster_list<<<dim3((unsigned)bx, (unsigned)nb), 256, 0, s>>>(V, faces, F, ncl, list, count, cams, frame0, H, W,
                                                                   keys);
}

void launch_resolve(unsigned long long *keys, int nb, int H, int W, const int32_t *row0, const int32_t *texinfo,
                    const float4 *V, const int4 *faces, const Camera *cams, int frame0, int32_t *idmap,
                    int32_t *idmap2, cudaStream_t s)
{
    const int64_t total = (int64_t)nb * H * W;
    if (total <= 0) return;
    const unsigned g = (unsigned)((total + kPixPerBlock - 1) / kPixPerBlock);
    if (row0)
        k_resolve<true><<<g, kPixThreads, 0, s>>>(keys, total, H, W, row0, texinfo, V, faces, cams, frame0, idmap,
                                                    idmap2);
    else
        k_resolve<false><<<g, kPixThreads, 0, s>>>(keys, total, H, W, row0, texinfo, V, faces, cams, frame0, idmap,
                                                     idmap2);
}

}  // namespace lf
