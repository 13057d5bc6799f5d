// Device-side raster rules shared by the raster kernels and the fused
// scatter (Sec. 3.3.1): camera-space transform and 1/256-pixel snap of a
// vertex, triangle set-up with orientation fix-up, and the bounding-box walk that tests every pixel centre with
// integer edge functions (top-left fill rule) and keeps the nearest surface
// per pixel with a 64-bit atomicMin of ((0xFFFFFFFF - bits(1/z)) << 32 | triangle).
//
// Determinism: every floating-point step uses explicit round-to-nearest
// intrinsics, which the compiler never contracts into FMAs, so the integer
// decisions are the same on every run and in every kernel that uses them.
#pragma once

#include "lf_internal.cuh"
#include "ptx.cuh"

namespace lf {

__device__ __forceinline__ float fmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fdiv(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ float i2f(long long v) { return __ll2float_rn(v); }

// Camera-space transform of a vertex in binary32 with a fixed operation
// order: X, Y = image x, y times the depth, in 1/256-pixel units; Z = depth.
__device__ __forceinline__ void transform_vertex(const float *A, float4 p, float &X, float &Y, float &Z)
{
    X = fadd(fadd(fadd(fmul(A[0], p.x), fmul(A[1], p.y)), fmul(A[2], p.z)), A[3]);
    Y = fadd(fadd(fadd(fmul(A[4], p.x), fmul(A[5], p.y)), fmul(A[6], p.z)), A[7]);
    Z = fadd(fadd(fadd(fmul(A[8], p.x), fmul(A[9], p.y)), fmul(A[10], p.z)), A[11]);
}

// Snaps a transformed vertex (Z > near plane): xs = rint(X / Z), ys =
// rint(Y / Z) with correctly rounded quotients, iz = RN(1 / Z); false if
// outside the snap range (the triangle is then dropped).  The quotients come
// from one correctly rounded reciprocal y = RN(1 / Z) by Markstein's
// correction (P. Markstein, IBM J. Res. Dev. 34(1), 1990): q = RN(a y), the
// exact remainder r = a - Z q (one FMA), RN(q + r y) = RN(a / Z) for
// quotients in the normal range; a smaller quotient snaps to 0 either way.
__device__ __forceinline__ bool snap_vertex(float X, float Y, float Z, int &xs, int &ys, float &iz)
{
    const float y = __frcp_rn(Z);
    const float qx = fmul(X, y), qy = fmul(Y, y);
    const float xf = __fmaf_rn(__fmaf_rn(-Z, qx, X), y, qx);
    const float yf = __fmaf_rn(__fmaf_rn(-Z, qy, Y), y, qy);
    if (!(fabsf(xf) <= kSnapLimit) || !(fabsf(yf) <= kSnapLimit)) return false;
    xs = __float2int_rn(xf);
    ys = __float2int_rn(yf);
    iz = y;
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

// Set-up of face f: false if it draws nothing (a vertex at or behind the
// near plane, outside the snap range, or zero area).  With an image size
// (W > 0), a face whose three vertices all lie more than 2 pixels beyond the
// same image side is dropped before its divisions: its bounding box misses
// the image, so nothing changes (the quotients round monotonically, and the
// side bounds are exact or dwarf their rounding).
__device__ __forceinline__ bool setup_triangle(const float *A, const float4 *__restrict__ V, int4 f, Tri &t,
                                               int H = 0, int W = 0)
{
    float X[3], Y[3], Z[3];
    transform_vertex(A, V[f.x], X[0], Y[0], Z[0]);
    transform_vertex(A, V[f.y], X[1], Y[1], Z[1]);
    transform_vertex(A, V[f.z], X[2], Y[2], Z[2]);
    if (!(Z[0] > kZNear) || !(Z[1] > kZNear) || !(Z[2] > kZNear)) return false;
    if (W > 0) {
        const float right = 256.0f * (float)(W + 1), bottom = 256.0f * (float)(H + 1);
        bool l = true, r = true, u = true, d = true;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            l = l && X[k] < -512.0f * Z[k];
            r = r && X[k] > right * Z[k];
            u = u && Y[k] < -512.0f * Z[k];
            d = d && Y[k] > bottom * Z[k];
        }
        if (l || r || u || d) return false;
    }
#pragma unroll
    for (int k = 0; k < 3; ++k)
        if (!snap_vertex(X[k], Y[k], Z[k], t.x[k], t.y[k], t.iz[k])) return false;
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
        tl[k] = top_left(t, k);
        // inside iff every value + its fill-rule bias > 0, i.e. value >= 1 - bias
        e_row[k] = dx * ((T)256 * y0 - t.y[bb]) - dy * ((T)256 * x0 - t.x[bb]);
        sx[k] = (T)-256 * dy;
        sy[k] = (T)256 * dx;
    }
    // inv_z = RN(num / area2) by Markstein's correction (P. Markstein, IBM J.
    // Res. Dev. 34(1), 1990): with y = RN(1 / b) and q = RN(a y), the exact
    // remainder r = a - b q (one FMA) gives RN(a / b) = RN(q + r y) for
    // normal, non-overflowing quotients -- here 1/z of a vertex in front of the
    // near plane.  One division per triangle instead of one per pixel.
    const float farea = i2f(t.area2);
    const float rcp = fdiv(1.0f, farea);
    const T th0 = (T)(1 - tl[0]), th1 = (T)(1 - tl[1]), th2 = (T)(1 - tl[2]);
    for (int py = y0; py <= y1; ++py) {
        T e0 = e_row[0], e1 = e_row[1], e2 = e_row[2];
        unsigned long long *row_keys = frame_keys + (int64_t)py * W;
        bool in_run = false;  // the covered samples of a row form one run (a convex face)
        for (int px = x0; px <= x1; ++px) {
            const bool inside = e0 >= th0 && e1 >= th1 && e2 >= th2;
            if (!inside && in_run) break;
            if (inside) {
                in_run = true;
                const float num = fadd(fadd(fmul(to_float(e0), t.iz[0]), fmul(to_float(e1), t.iz[1])),
                                       fmul(to_float(e2), t.iz[2]));
                const float q = fmul(num, rcp);
                const float inv_z = __fmaf_rn(__fmaf_rn(-farea, q, num), rcp, q);
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

// Conservative frustum test of one 32-face cluster for one frame (A: the
// frame's camera rows).  The 8 corners of the cluster's world box are
// evaluated in homogeneous image coordinates; if one affine bound is violated
// at all corners it is violated everywhere in the box: every vertex then
// projects more than 2 pixels left of / right of / above / below the image,
// or lies in front of the near plane, so the renderer drops every triangle of
// the cluster anyway.  The 2-pixel and 0.01 m margins dwarf the binary32
// evaluation error, so a culled cluster never holds a pixel.
__device__ __forceinline__ bool cluster_may_be_visible(const float4 *__restrict__ bounds, int64_t cl, const float *A,
                                                       int H, int W)
{
    const float4 lo = bounds[2 * cl], hi = bounds[2 * cl + 1];
    if (lo.w != 0.0f) return false;  // no valid face
    bool left = true, right = true, top = true, bottom = true, near = true;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const float px = (k & 1) ? hi.x : lo.x, py = (k & 2) ? hi.y : lo.y, pz = (k & 4) ? hi.z : lo.z;
        const float X = A[0] * px + A[1] * py + A[2] * pz + A[3];
        const float Y = A[4] * px + A[5] * py + A[6] * pz + A[7];
        const float Z = A[8] * px + A[9] * py + A[10] * pz + A[11];
        left = left && X + 512.0f * Z < 0.0f;
        right = right && X - 256.0f * (float)(W + 1) * Z > 0.0f;
        top = top && Y + 512.0f * Z < 0.0f;
        bottom = bottom && Y - 256.0f * (float)(H + 1) * Z > 0.0f;
        near = near && Z < kZNear - 0.01f;
    }
    return !(left || right || top || bottom || near);
}

// Set-up and box walk of face f for one frame (one thread per face; faces
// past F, dropped by the packer, or culled by set-up draw nothing).
__device__ __forceinline__ void raster_face(const float *A, const float4 *__restrict__ V,
                                            const int4 *__restrict__ faces, int64_t F, int64_t f, int H, int W,
                                            unsigned long long *__restrict__ frame_keys)
{
    if (f >= F) return;
    const int4 fc = faces[f];
    if (!fc.w) return;
    Tri t;
    if (!setup_triangle(A, V, fc, t, H, W)) return;
    int minx = min(t.x[0], min(t.x[1], t.x[2])), maxx = max(t.x[0], max(t.x[1], t.x[2]));
    int miny = min(t.y[0], min(t.y[1], t.y[2])), maxy = max(t.y[0], max(t.y[1], t.y[2]));
    int x0 = max(ceil256(minx), 0), x1 = min(floor256(maxx), W - 1);
    int y0 = max(ceil256(miny), 0), y1 = min(floor256(maxy), H - 1);
    if (x0 > x1 || y0 > y1) return;
    // Small triangles (extent <= 64 px, the common case) keep every edge
    // function value below 2^30 in magnitude, so the same integers are
    // stepped in 32 bits; larger ones use 64 bits.  Results are identical.
    if (maxx - minx <= (1 << 14) && maxy - miny <= (1 << 14))
        raster_box<int>(t, x0, x1, y0, y1, (unsigned int)f, frame_keys, W);
    else
        raster_box<long long>(t, x0, x1, y0, y1, (unsigned int)f, frame_keys, W);
}

}  // namespace lf
