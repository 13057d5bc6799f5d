// Renderer kernels (Sec. 3.3.1): per-frame camera set-up, triangle raster with
// a 64-bit z-buffer key, and the resolve of the z-buffer into row indices
// l = id_t + id_x (Eq. texel-in-array).
//
// Determinism: every floating-point step uses explicit round-to-nearest
// intrinsics (__fmul_rn, __fadd_rn, __fdiv_rn, __dmul_rn, __dadd_rn), which the
// compiler never contracts into FMAs, so the integer decisions (snapped vertex
// positions, coverage, the depth key) are the same on every run and match the
// project's raster reading bit for bit.
#include <mutex>

#include "lf_internal.cuh"
#include "ptx.cuh"

namespace lf {
namespace {

__device__ __forceinline__ float fmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fdiv(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ float i2f(long long v) { return __ll2float_rn(v); }

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

// Projects and snaps one vertex; false if it is at/behind the near plane or
// outside the snap range (its triangle is then dropped).
__device__ __forceinline__ bool project_vertex(const float *A, float4 p, int &xs, int &ys, float &iz)
{
    float X = fadd(fadd(fadd(fmul(A[0], p.x), fmul(A[1], p.y)), fmul(A[2], p.z)), A[3]);
    float Y = fadd(fadd(fadd(fmul(A[4], p.x), fmul(A[5], p.y)), fmul(A[6], p.z)), A[7]);
    float Z = fadd(fadd(fadd(fmul(A[8], p.x), fmul(A[9], p.y)), fmul(A[10], p.z)), A[11]);
    if (!(Z > kZNear)) return false;
    float xf = fdiv(X, Z);
    float yf = fdiv(Y, Z);
    if (!(fabsf(xf) <= kSnapLimit) || !(fabsf(yf) <= kSnapLimit)) return false;
    xs = __float2int_rn(xf);
    ys = __float2int_rn(yf);
    iz = fdiv(1.0f, Z);
    return true;
}

// Screen-space triangle after orientation fix-up: positive area, so each edge
// function is >= 0 inside.  perm[k] = original local index of vertex k.
struct Tri {
    int x[3], y[3];
    float iz[3];
    long long area2;
    bool swapped;
};

__device__ __forceinline__ bool setup_triangle(const float *A, const float4 *__restrict__ V, int4 f, Tri &t)
{
    if (!project_vertex(A, V[f.x], t.x[0], t.y[0], t.iz[0])) return false;
    if (!project_vertex(A, V[f.y], t.x[1], t.y[1], t.iz[1])) return false;
    if (!project_vertex(A, V[f.z], t.x[2], t.y[2], t.iz[2])) return false;
    long long area2 = (long long)(t.x[1] - t.x[0]) * (t.y[2] - t.y[0]) - (long long)(t.y[1] - t.y[0]) * (t.x[2] - t.x[0]);
    if (area2 == 0) return false;
    t.swapped = area2 < 0;
    if (t.swapped) {
        int tx = t.x[1], ty = t.y[1];
        float tz = t.iz[1];
        t.x[1] = t.x[2];
        t.y[1] = t.y[2];
        t.iz[1] = t.iz[2];
        t.x[2] = tx;
        t.y[2] = ty;
        t.iz[2] = tz;
        area2 = -area2;
    }
    t.area2 = area2;
    return true;
}

// Edge function of vertex k (edge b -> c opposite it) at sample (px, py).
__device__ __forceinline__ long long edge_at(const Tri &t, int k, long long px, long long py)
{
    const int b = (k + 1) % 3, c = (k + 2) % 3;
    long long dx = t.x[c] - t.x[b], dy = t.y[c] - t.y[b];
    return dx * (py - t.y[b]) - dy * (px - t.x[b]);
}

// Top-left rule in y-down image coordinates: an edge direction with dy < 0
// is a left edge, dy == 0 && dx > 0 a top edge; samples on them are inside.
__device__ __forceinline__ int top_left(const Tri &t, int k)
{
    const int b = (k + 1) % 3, c = (k + 2) % 3;
    int dx = t.x[c] - t.x[b], dy = t.y[c] - t.y[b];
    return (dy < 0 || (dy == 0 && dx > 0)) ? 1 : 0;
}

__device__ __forceinline__ int floor256(int a) { return a >> 8; }        // arithmetic shift = floor
__device__ __forceinline__ int ceil256(int a) { return -((-a) >> 8); }

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

// Conservative frustum test of one cluster (whole warp, uniform result):
// true when no triangle of the cluster can cover a pixel centre of this
// frame.  Each of the box's 8 corners is evaluated in homogeneous image
// coordinates; if one affine bound is violated at all corners it is violated
// everywhere in the box: every vertex then projects more than 2 pixels left
// of / right of / above / below the image, or lies in front of the near
// plane (so every triangle is dropped by the renderer anyway).  The 2-pixel
// and 0.01 m margins dwarf the binary32 evaluation error of this test.
__device__ __forceinline__ bool cluster_culled(const float *A, const float4 *__restrict__ bounds, int64_t cl, int H,
                                               int W, int lane)
{
    const float4 lo = bounds[2 * cl], hi = bounds[2 * cl + 1];
    if (lo.w != 0.0f) return true;
    const float px = (lane & 1) ? hi.x : lo.x, py = (lane & 2) ? hi.y : lo.y, pz = (lane & 4) ? hi.z : lo.z;
    const float X = A[0] * px + A[1] * py + A[2] * pz + A[3];
    const float Y = A[4] * px + A[5] * py + A[6] * pz + A[7];
    const float Z = A[8] * px + A[9] * py + A[10] * pz + A[11];
    const bool corner = lane < 8;
    const bool left = !corner || X + 512.0f * Z < 0.0f;
    const bool right = !corner || X - 256.0f * (float)(W + 1) * Z > 0.0f;
    const bool top = !corner || Y + 512.0f * Z < 0.0f;
    const bool bottom = !corner || Y - 256.0f * (float)(H + 1) * Z > 0.0f;
    const bool near = !corner || Z < kZNear - 0.01f;
    return __all_sync(0xffffffffu, left) || __all_sync(0xffffffffu, right) || __all_sync(0xffffffffu, top) ||
           __all_sync(0xffffffffu, bottom) || __all_sync(0xffffffffu, near);
}

__device__ __forceinline__ float to_float(int v) { return __int2float_rn(v); }
__device__ __forceinline__ float to_float(long long v) { return __ll2float_rn(v); }

// Tests every pixel centre of the clamped box [x0, x1] x [y0, y1] with edge
// functions stepped incrementally in integer type T; covered samples take a
// 64-bit atomicMin of ((0xFFFFFFFF - bits(1/z)) << 32 | triangle).
template <typename T>
__device__ __forceinline__ void raster_box(const Tri &t, int x0, int x1, int y0, int y1, unsigned int fid,
                                           unsigned long long *__restrict__ frame_keys, int W)
{
    T e_row[3], sx[3], sy[3];
    int tl[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int bb = (k + 1) % 3, cc = (k + 2) % 3;
        const T dx = (T)(t.x[cc] - t.x[bb]), dy = (T)(t.y[cc] - t.y[bb]);
        e_row[k] = dx * ((T)256 * y0 - t.y[bb]) - dy * ((T)256 * x0 - t.x[bb]);
        sx[k] = (T)-256 * dy;
        sy[k] = (T)256 * dx;
        tl[k] = top_left(t, k);
    }
    const float farea = i2f(t.area2);
    for (int py = y0; py <= y1; ++py) {
        T e0 = e_row[0], e1 = e_row[1], e2 = e_row[2];
        unsigned long long *row_keys = frame_keys + (int64_t)py * W;
        for (int px = x0; px <= x1; ++px) {
            if (e0 + tl[0] > 0 && e1 + tl[1] > 0 && e2 + tl[2] > 0) {
                const float num =
                    fadd(fadd(fmul(to_float(e0), t.iz[0]), fmul(to_float(e1), t.iz[1])), fmul(to_float(e2), t.iz[2]));
                const float inv_z = fdiv(num, farea);
                const unsigned long long key = ((unsigned long long)(0xFFFFFFFFu - __float_as_uint(inv_z)) << 32) | fid;
                red_min_u64(row_keys + px, key);
            }
            e0 += sx[0];
            e1 += sx[1];
            e2 += sx[2];
        }
        e_row[0] += sy[0];
        e_row[1] += sy[1];
        e_row[2] += sy[2];
    }
}

// One warp per cluster of 32 faces and one thread per face, for one frame:
// conservative cluster cull, then per triangle set-up; every pixel centre of
// the clamped bounding box is tested with incrementally stepped int64 edge
// functions; covered samples take a 64-bit atomicMin of
// ((0xFFFFFFFF - bits(1/z)) << 32 | triangle) into the frame's z-buffer.
__global__ void __launch_bounds__(256, 4) k_raster(const float4 *__restrict__ V, const int4 *__restrict__ faces,
                                                int64_t F, const float4 *__restrict__ bounds,
                                                const Camera *__restrict__ cams, int frame0, int H, int W,
                                                unsigned long long *__restrict__ keys)
{
    __shared__ float A[12];
    const int b = blockIdx.y;
    if (threadIdx.x < 12) A[threadIdx.x] = cams[frame0 + b].a[threadIdx.x];
    __syncthreads();
    const int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t cl = f / kClusterFaces;
    if (cl * kClusterFaces >= F) return;  // whole warp past the end
    if (cluster_culled(A, bounds, cl, H, W, threadIdx.x & 31)) return;
    if (f >= F) return;
    const int4 fc = faces[f];
    if (!fc.w) return;
    Tri t;
    if (!setup_triangle(A, V, fc, t)) return;
    int minx = min(t.x[0], min(t.x[1], t.x[2])), maxx = max(t.x[0], max(t.x[1], t.x[2]));
    int miny = min(t.y[0], min(t.y[1], t.y[2])), maxy = max(t.y[0], max(t.y[1], t.y[2]));
    int x0 = max(ceil256(minx), 0), x1 = min(floor256(maxx), W - 1);
    int y0 = max(ceil256(miny), 0), y1 = min(floor256(maxy), H - 1);
    if (x0 > x1 || y0 > y1) return;

    const unsigned int fid = (unsigned int)f;
    unsigned long long *frame_keys = keys + (int64_t)b * H * W;
    // Small triangles (extent <= 64 px, the common case) keep every edge
    // function value below 2^30 in magnitude, so the same integers are
    // stepped in 32 bits; larger ones use 64 bits.  Results are identical.
    if (maxx - minx <= (1 << 14) && maxy - miny <= (1 << 14))
        raster_box<int>(t, x0, x1, y0, y1, fid, frame_keys, W);
    else
        raster_box<long long>(t, x0, x1, y0, y1, fid, frame_keys, W);
}

// z-buffer -> row map, and re-arms the z-buffer for the next batch.  For a
// subdivided triangle (s > 1) the winning triangle's perspective-correct
// barycentrics are recomputed with the same operations as the raster:
// beta_k = (float)E_k * iz_k / ((w0 + w1) + w2); u, v are the barycentrics of
// the vertices after the uv origin; the texel cell (i, j) is
// (floor(s u), floor(s v)) clamped into the triangle and id_x = T(i + j) + j.
__global__ void __launch_bounds__(256) k_resolve(unsigned long long *__restrict__ keys, int64_t total, int H, int W,
                                                 const int32_t *__restrict__ row0,
                                                 const int32_t *__restrict__ texinfo,
                                                 const float4 *__restrict__ V, const int4 *__restrict__ faces,
                                                 const Camera *__restrict__ cams, int frame0,
                                                 int32_t *__restrict__ idmap, int32_t *__restrict__ idmap2)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= total) return;
    const unsigned long long key = keys[p];
    keys[p] = kEmptyKey;
    int32_t row = -1;
    if (key != kEmptyKey) {
        const int f = (int)(unsigned int)key;
        if (!row0) {
            row = f;
        } else {
            const int info = texinfo[f];
            const int s = info & 0xFFFF;
            const int o = info >> 16;
            int idx = 0;
            if (s > 1) {
                const int64_t npix = (int64_t)H * W;
                const int b = (int)(p / npix);
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
            row = row0[f] + idx;
        }
    }
    idmap[p] = row;
    if (idmap2) idmap2[p] = row;
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
    if (!setup_triangle(A, P, make_int4(0, 1, 2, 1), t)) return;
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
// device address once per device (below).
static __device__ __align__(256) unsigned long long
    g_noalloc_scratch[SM_NOALLOC_MAX_PIXELS + 6 * SM_NOALLOC_MAX_FRAMES];

namespace {
std::mutex g_noalloc_mu;
unsigned long long *g_noalloc_ptr[64] = {};  // device address of the scratch, per device ordinal
}  // namespace

// Device address of the static scratch on the current device; the first call
// on a device looks it up (cudaGetSymbolAddress, which needs that device
// current and allocates nothing).
cudaError_t noalloc_scratch(unsigned long long **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_ptr[dev] = static_cast<unsigned long long *>(p);
    }
    *out = g_noalloc_ptr[dev];
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
        k_resolve<<<(unsigned)((npix + 255) / 256), 256, 0, s>>>(keys, npix, H, W, nullptr, nullptr, nullptr, nullptr,
                                                                  cams, i, idmap + (int64_t)i * npix, nullptr);
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
                   int frame0, int nb, int H, int W, unsigned long long *keys, cudaStream_t s)
{
    if (F <= 0 || nb <= 0) return;
    dim3 grid((unsigned)((F + 255) / 256), (unsigned)nb);
    k_raster<<<grid, 256, 0, s>>>(V, faces, F, bounds, cams, frame0, H, W, keys);
}

void launch_resolve(unsigned long long *keys, int nb, int H, int W, const int32_t *row0, const int32_t *texinfo,
                    const float4 *V, const int4 *faces, const Camera *cams, int frame0, int32_t *idmap,
                    int32_t *idmap2, cudaStream_t s)
{
    const int64_t total = (int64_t)nb * H * W;
    if (total <= 0) return;
    k_resolve<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(keys, total, H, W, row0, texinfo, V, faces, cams,
                                                                frame0, idmap, idmap2);
}

}  // namespace lf
