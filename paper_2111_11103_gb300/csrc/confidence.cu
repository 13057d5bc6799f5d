// Learned per-observation confidence: an extension of the weighted fusion
// rules (Sec. 3.2.2, Eqs. w-sum / w-mul / w-maxsum), where the weight of an
// observation comes from a small network instead of being 1 or
// 1/|K_i ∩ K_x|.
//
//  * k_conf_features: per pixel of a rasterised batch, five features -- |cos|
//    between the visible triangle's normal and the pixel's viewing ray, depth
//    (1 / interpolated 1/z, / 4 m), prediction entropy (/ ln c), top-2
//    margin, distance to the image border (/ half the smaller side).
//  * k_conf_forward: 5 -> 32 -> 32 -> 1 MLP, ReLU, the parameters rounded to
//    bfloat16, float32 accumulation.  Its output o is the log-odds that the
//    observation agrees with the fused label (trained with the binary
//    cross-entropy of sigmoid(o)); the fusion weight is w = max(o, 1/16),
//    the optimal weight of an independent two-way vote (Nitzan and Paroush,
//    1982) clipped at a small floor, so that a row whose every observation
//    is predicted below even odds keeps the plain vote instead of a tie.
//  * k_conf_grad + k_conf_update: one step of gradient descent on the mean
//    binary cross-entropy; each block reduces its observations' gradients in
//    shared memory (fixed order), converts the sums to 64-bit fixed point
//    (2^-40) and adds them with integer atomics, so the step's gradient does
//    not depend on the order in which blocks finish: training runs are
//    reproducible bit for bit.
//  * k_conf_targets: 1 where a pixel's arg max equals its row's fused label.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "lf_internal.cuh"

namespace lf {

constexpr float kWeightFloor = 0.0625f;  // 1/16: the least fusion weight of an observation
namespace {

constexpr int kF = SM_CONF_FEATURES;  // 5
constexpr int kH = 32;                 // hidden width
// parameter offsets: W1 (kH x kF, row = output), b1, W2 (kH x kH), b2, w3, b3
constexpr int kW1 = 0, kB1 = kW1 + kH * kF, kW2 = kB1 + kH, kB2 = kW2 + kH * kH, kW3 = kB2 + kH, kB3 = kW3 + kH;
static_assert(kB3 + 1 == SM_CONF_PARAMS, "parameter layout");
constexpr float kPMin = 9.313225746154785e-10f;  // 2^-30

__device__ __forceinline__ float load_p(const void *probs, sm_dtype dt, int64_t i, float sc)
{
    if (dt == SM_F32) return static_cast<const float *>(probs)[i];
    if (dt == SM_BF16) {
        const unsigned short u = static_cast<const unsigned short *>(probs)[i];
        return __fmul_rn(__uint_as_float((unsigned)u << 16), sc);
    }
    __half_raw h = __nv_cvt_fp8_to_halfraw(static_cast<const __nv_fp8_storage_t *>(probs)[i], __NV_E4M3);
    return __fmul_rn(__half2float(*reinterpret_cast<__half *>(&h)), sc);
}

__global__ void __launch_bounds__(256)
    k_conf_features(const unsigned long long *__restrict__ keys, int64_t total, int H, int W,
                    const float4 *__restrict__ V, const int4 *__restrict__ faces, int64_t F,
                    const sm_intrinsics *__restrict__ K, const double *__restrict__ T, const void *__restrict__ probs,
                    sm_dtype dt, const float *__restrict__ scale, int c, float *__restrict__ feat)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= total) return;
    const int64_t npix = (int64_t)H * W;
    const int b = (int)frame_of(p, npix);
    const int64_t q = p - (int64_t)b * npix;
    const int y = (int)(q / W), x = (int)(q - (int64_t)y * W);
    float *out = feat + p * kF;
    const unsigned long long key = keys[p];
    const int64_t f = (int64_t)(unsigned int)key;
    if (key == kEmptyKey || f >= F) {
        for (int k = 0; k < kF; ++k) out[k] = 0.0f;
        return;
    }
    // viewing ray in world coordinates: R_cw ((x - cx) / fx, (y - cy) / fy, 1)
    const sm_intrinsics Kb = K[b];
    const double *Tb = T + 16 * (int64_t)b;
    const float dx = ((float)x - (float)Kb.cx) / (float)Kb.fx, dy = ((float)y - (float)Kb.cy) / (float)Kb.fy;
    float ray[3];
    for (int r = 0; r < 3; ++r) ray[r] = (float)Tb[4 * r] * dx + (float)Tb[4 * r + 1] * dy + (float)Tb[4 * r + 2];
    const int4 fc = faces[f];
    const float4 a = V[fc.x], bb = V[fc.y], cc = V[fc.z];
    const float e1[3] = {bb.x - a.x, bb.y - a.y, bb.z - a.z}, e2[3] = {cc.x - a.x, cc.y - a.y, cc.z - a.z};
    const float n[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
    const float dot = n[0] * ray[0] + n[1] * ray[1] + n[2] * ray[2];
    const float nn = sqrtf(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    const float rr = sqrtf(ray[0] * ray[0] + ray[1] * ray[1] + ray[2] * ray[2]);
    out[0] = nn > 0.0f ? fabsf(dot) / (nn * rr) : 0.0f;
    const float inv_z = __uint_as_float(0xFFFFFFFFu - (unsigned int)(key >> 32));
    out[1] = inv_z > 0.0f ? 0.25f / inv_z : 0.0f;
    // entropy and top-2 margin of the prediction
    const float sc = (dt == SM_F32) ? 1.0f : scale[p];
    float ent = 0.0f, m1 = -INFINITY, m2 = -INFINITY;
    for (int j = 0; j < c; ++j) {
        const float v = load_p(probs, dt, p * c + j, sc);
        ent -= v * logf(fmaxf(v, kPMin));
        if (v > m1) {
            m2 = m1;
            m1 = v;
        } else if (v > m2) {
            m2 = v;
        }
    }
    out[2] = c > 1 ? ent / logf((float)c) : 0.0f;
    out[3] = c > 1 ? m1 - m2 : m1;
    const int d = min(min(x, y), min(W - 1 - x, H - 1 - y));
    out[4] = (float)d / (0.5f * (float)min(W, H));
}

// Parameters rounded to bfloat16, in shared memory.
__device__ __forceinline__ void load_params(const float *__restrict__ params, float *s)
{
    for (int i = threadIdx.x; i < SM_CONF_PARAMS; i += blockDim.x)
        s[i] = __bfloat162float(__float2bfloat16_rn(params[i]));
    __syncthreads();
}

// Forward pass of one observation; z1, z2: pre-activations.
__device__ __forceinline__ float mlp_forward(const float *s, const float *x, float *z1, float *z2)
{
    float h1[kH];
#pragma unroll
    for (int i = 0; i < kH; ++i) {
        float acc = s[kB1 + i];
#pragma unroll
        for (int k = 0; k < kF; ++k) acc = fmaf(s[kW1 + i * kF + k], x[k], acc);
        z1[i] = acc;
        h1[i] = fmaxf(acc, 0.0f);
    }
    float o = s[kB3];
#pragma unroll 4
    for (int j = 0; j < kH; ++j) {
        float acc = s[kB2 + j];
#pragma unroll
        for (int i = 0; i < kH; ++i) acc = fmaf(s[kW2 + j * kH + i], h1[i], acc);
        z2[j] = acc;
        o = fmaf(s[kW3 + j], fmaxf(acc, 0.0f), o);
    }
    return o;
}

// ---- inference fused with the features, hidden layer on the tensor cores ----

// Two floats rounded to bfloat16 (nearest even) and packed, the first in the
// low half (the element with the lower column index of an mma fragment).
__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi)
{
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&v);
}

// D = A B + C for one 16 x 8 x 16 tile: A 16 x 16 bfloat16 (row major), B
// 16 x 8 bfloat16 (column major), C and D float32; fragments as the PTX ISA
// lays them out for mma.m16n8k16 (g = lane / 4, t = lane % 4): a0 (row g,
// cols 2t, 2t+1), a1 (row g+8, same cols), a2 / a3 (cols + 8); b0 (rows 2t,
// 2t+1, col g), b1 (rows + 8); c0, c1 (row g, cols 2t, 2t+1), c2, c3 (row g+8).
__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2])
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Features of pixel p of a rasterised batch (see k_conf_features), from its
// z-buffer key; false for background.
__device__ __forceinline__ bool pixel_features(unsigned long long key, int64_t p, int H, int W,
                                               const float4 *__restrict__ V, const int4 *__restrict__ faces, int64_t F,
                                               const sm_intrinsics *__restrict__ K, const double *__restrict__ T,
                                               const void *__restrict__ probs, sm_dtype dt,
                                               const float *__restrict__ scale, int c, float (&x)[kF])
{
    const int64_t npix = (int64_t)H * W;
    const int b = (int)frame_of(p, npix);
    const int64_t q = p - (int64_t)b * npix;
    const int y = (int)(q / W), xx = (int)(q - (int64_t)y * W);
    const int64_t f = (int64_t)(unsigned int)key;
    if (key == kEmptyKey || f >= F) return false;
    const sm_intrinsics Kb = K[b];
    const double *Tb = T + 16 * (int64_t)b;
    const float dx = ((float)xx - (float)Kb.cx) / (float)Kb.fx, dy = ((float)y - (float)Kb.cy) / (float)Kb.fy;
    float ray[3];
    for (int r = 0; r < 3; ++r) ray[r] = (float)Tb[4 * r] * dx + (float)Tb[4 * r + 1] * dy + (float)Tb[4 * r + 2];
    const int4 fc = faces[f];
    const float4 a = V[fc.x], bb = V[fc.y], cc = V[fc.z];
    const float e1[3] = {bb.x - a.x, bb.y - a.y, bb.z - a.z}, e2[3] = {cc.x - a.x, cc.y - a.y, cc.z - a.z};
    const float n[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
    const float dot = n[0] * ray[0] + n[1] * ray[1] + n[2] * ray[2];
    const float nn = sqrtf(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    const float rr = sqrtf(ray[0] * ray[0] + ray[1] * ray[1] + ray[2] * ray[2]);
    x[0] = nn > 0.0f ? fabsf(dot) / (nn * rr) : 0.0f;
    const float inv_z = __uint_as_float(0xFFFFFFFFu - (unsigned int)(key >> 32));
    x[1] = inv_z > 0.0f ? 0.25f / inv_z : 0.0f;
    const float sc = (dt == SM_F32) ? 1.0f : scale[p];
    // entropy (hardware base-2 logarithm; its error, ~2^-22 relative, is far
    // below the bfloat16 rounding of the network's hidden layer) and top-2
    // margin, four classes per load when the pixel's row is 16-byte aligned.
    // BF16 / FP8: on the codes q = p / s, the scale applied once:
    // -sum p log2 p = -s (sum q log2 q + log2(s) sum q), the margin is s times
    // the codes' margin (the clamp at 2^-30 / s keeps the entropy's terms
    // those of p, up to rounding)
    const bool coded = dt != SM_F32 && sc > 0.0f;  // a zero scale means an all-zero prediction
    const float qmin = coded ? kPMin / sc : kPMin;
    float eq = 0.0f, sq = 0.0f, m1 = -INFINITY, m2 = -INFINITY;
    auto take = [&](float v) {
        eq = fmaf(v, __log2f(fmaxf(v, qmin)), eq);
        sq += v;
        if (v > m1) {
            m2 = m1;
            m1 = v;
        } else if (v > m2) {
            m2 = v;
        }
    };
    const int esz = dt == SM_F32 ? 4 : (dt == SM_BF16 ? 2 : 1);
    const uint8_t *row = static_cast<const uint8_t *>(probs) + (size_t)p * c * esz;
    if ((c & 3) == 0 && ((uintptr_t)row & (4 * esz - 1)) == 0) {
        for (int j = 0; j < c; j += 4) {
            if (dt == SM_F32) {
                const float4 q = *reinterpret_cast<const float4 *>(row + 4 * j);
                take(q.x); take(q.y); take(q.z); take(q.w);
            } else if (dt == SM_BF16) {
                const uint2 u = *reinterpret_cast<const uint2 *>(row + 2 * j);
                take(__uint_as_float(u.x << 16)); take(__uint_as_float(u.x & 0xffff0000u));
                take(__uint_as_float(u.y << 16)); take(__uint_as_float(u.y & 0xffff0000u));
            } else {
                const uint32_t u = *reinterpret_cast<const uint32_t *>(row + j);
                __half2_raw lo = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(u & 0xffffu), __NV_E4M3);
                __half2_raw hi = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(u >> 16), __NV_E4M3);
                const float2 a2 = __half22float2(*reinterpret_cast<__half2 *>(&lo));
                const float2 b2 = __half22float2(*reinterpret_cast<__half2 *>(&hi));
                take(a2.x); take(a2.y); take(b2.x); take(b2.y);
            }
        }
    } else {
        for (int j = 0; j < c; ++j) take(load_p(probs, dt, p * c + j, 1.0f));
    }
    const float ent2 = coded ? -sc * fmaf(__log2f(sc), sq, eq) : (dt == SM_F32 ? -eq : 0.0f);
    x[2] = c > 1 ? ent2 / __log2f((float)c) : 0.0f;
    x[3] = c > 1 ? sc * (m1 - m2) : sc * m1;
    const int d = min(min(xx, y), min(W - 1 - xx, H - 1 - y));
    x[4] = (float)d / (0.5f * (float)min(W, H));
    return true;
}

// One thread per pixel of a rasterised batch, one warp per 32 pixels: the
// features, then w = max(network, 1/16) with the bfloat16 parameters; the
// first layer in float32, the 32 x 32 hidden layer as 16 tensor-core tiles
// per warp (activations rounded to bfloat16, float32 accumulation), the
// output layer in float32.  Writes w (0 for background) and, when rows_out
// is given, the triangle of every pixel (-1 for background), re-arming the
// z-buffer; without rows_out the keys are left as they are.
__global__ void __launch_bounds__(256)
    k_conf_weights(unsigned long long *__restrict__ keys, int64_t total, int H, int W, const float4 *__restrict__ V,
                   const int4 *__restrict__ faces, int64_t F, const sm_intrinsics *__restrict__ K,
                   const double *__restrict__ T, const void *__restrict__ probs, sm_dtype dt,
                   const float *__restrict__ scale, int c, const float *__restrict__ params, float *__restrict__ w_out,
                   int32_t *__restrict__ rows_out)
{
    __shared__ float s[SM_CONF_PARAMS];
    __shared__ __align__(16) __nv_bfloat16 hs[8][32][kH + 8];  // per warp: its 32 pixels' activations (padded rows)
    __shared__ __align__(16) __nv_bfloat16 w2[kH][kH + 8];     // W2 (row = output), bfloat16
    __shared__ float4 l1a[kH];                                   // first layer, unit i: W1[i][0..3]
    __shared__ float2 l1b[kH];                                   // W1[i][4], b1[i]
    load_params(params, s);
    for (int i = threadIdx.x; i < kH * kH; i += blockDim.x) w2[i / kH][i % kH] = __float2bfloat16_rn(s[kW2 + i]);
    for (int i = threadIdx.x; i < kH; i += blockDim.x) {
        l1a[i] = make_float4(s[kW1 + i * kF], s[kW1 + i * kF + 1], s[kW1 + i * kF + 2], s[kW1 + i * kF + 3]);
        l1b[i] = make_float2(s[kW1 + i * kF + 4], s[kB1 + i]);
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    // B fragments of W2^T for the 4 output tiles x 2 input steps (loaded once)
    uint32_t bf[4][2][2];
#pragma unroll
    for (int nt = 0; nt < 4; ++nt)
#pragma unroll
        for (int ks = 0; ks < 2; ++ks) {
            bf[nt][ks][0] = *reinterpret_cast<const uint32_t *>(&w2[8 * nt + g][16 * ks + 2 * t]);
            bf[nt][ks][1] = *reinterpret_cast<const uint32_t *>(&w2[8 * nt + g][16 * ks + 8 + 2 * t]);
        }
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + warp * 32; base < total; base += stride) {
        const int64_t p = base + lane;
        float x[kF] = {0.f, 0.f, 0.f, 0.f, 0.f};
        bool fg = false;
        int32_t row = -1;
        if (p < total) {
            const unsigned long long key = keys[p];
            fg = pixel_features(key, p, H, W, V, faces, F, K, T, probs, dt, scale, c, x);
            if (rows_out) {  // else the keys stay for the scatter or the resolve pass
                keys[p] = kEmptyKey;
                if (fg) row = (int32_t)(unsigned int)key;
                rows_out[p] = row;
            }
        }
        // first layer, float32, into this lane's row of activations
#pragma unroll
        for (int i = 0; i < kH; i += 2) {
            float z[2];
#pragma unroll
            for (int u = 0; u < 2; ++u) {  // b1 + W1 x in the order k = 0 .. 4
                const float4 a = l1a[i + u];
                const float2 b = l1b[i + u];
                z[u] = fmaf(b.x, x[4], fmaf(a.w, x[3], fmaf(a.z, x[2], fmaf(a.y, x[1], fmaf(a.x, x[0], b.y)))));
            }
            *reinterpret_cast<uint32_t *>(&hs[warp][lane][i]) = pack_bf16x2(fmaxf(z[0], 0.f), fmaxf(z[1], 0.f));
        }
        __syncwarp();
        // hidden layer: 32 pixels x 32 outputs = 2 x 4 tiles, K = 32 in 2 steps
        float o[2][2] = {{s[kB3], s[kB3]}, {s[kB3], s[kB3]}};  // per m tile: rows g and g + 8
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
            uint32_t af[2][4];
#pragma unroll
            for (int ks = 0; ks < 2; ++ks) {
                af[ks][0] = *reinterpret_cast<const uint32_t *>(&hs[warp][16 * mt + g][16 * ks + 2 * t]);
                af[ks][1] = *reinterpret_cast<const uint32_t *>(&hs[warp][16 * mt + g + 8][16 * ks + 2 * t]);
                af[ks][2] = *reinterpret_cast<const uint32_t *>(&hs[warp][16 * mt + g][16 * ks + 8 + 2 * t]);
                af[ks][3] = *reinterpret_cast<const uint32_t *>(&hs[warp][16 * mt + g + 8][16 * ks + 8 + 2 * t]);
            }
            float part[2] = {0.f, 0.f};
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) {
                const int j = 8 * nt + 2 * t;  // this thread's two output columns
                float d[4] = {s[kB2 + j], s[kB2 + j + 1], s[kB2 + j], s[kB2 + j + 1]};
                mma_bf16_16816(d, af[0], bf[nt][0]);
                mma_bf16_16816(d, af[1], bf[nt][1]);
                // output layer: w3 . relu(z2), this thread's columns
                part[0] = fmaf(s[kW3 + j], fmaxf(d[0], 0.f), part[0]);
                part[0] = fmaf(s[kW3 + j + 1], fmaxf(d[1], 0.f), part[0]);
                part[1] = fmaf(s[kW3 + j], fmaxf(d[2], 0.f), part[1]);
                part[1] = fmaf(s[kW3 + j + 1], fmaxf(d[3], 0.f), part[1]);
            }
            // sum over the 4 threads of the group (all 32 columns)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                part[h] += __shfl_xor_sync(0xffffffffu, part[h], 1);
                part[h] += __shfl_xor_sync(0xffffffffu, part[h], 2);
                o[mt][h] += part[h];
            }
        }
        // pixel 16 mt + g (+ 8) of the warp: its lane fetches the output from
        // thread 4 g of the group (the lanes own rows g and g + 8 of each tile)
        const int mt = lane >> 4, r = lane & 15;
        const int src = 4 * (r & 7);
        const float o0 = __shfl_sync(0xffffffffu, o[0][0], src), o1 = __shfl_sync(0xffffffffu, o[0][1], src);
        const float o2 = __shfl_sync(0xffffffffu, o[1][0], src), o3 = __shfl_sync(0xffffffffu, o[1][1], src);
        const float ol = mt == 0 ? (r < 8 ? o0 : o1) : (r < 8 ? o2 : o3);
        if (p < total) w_out[p] = fg ? fmaxf(ol, kWeightFloor) : 0.0f;
        __syncwarp();  // the activations are rewritten by the next pixels
    }
}

__global__ void __launch_bounds__(256)
    k_conf_forward(const float *__restrict__ params, const float *__restrict__ feat, int64_t n, float *__restrict__ w)
{
    __shared__ float s[SM_CONF_PARAMS];
    load_params(params, s);
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float x[kF], z1[kH], z2[kH];
#pragma unroll
    for (int k = 0; k < kF; ++k) x[k] = feat[i * kF + k];
    const float o = mlp_forward(s, x, z1, z2);
    w[i] = fmaxf(o, kWeightFloor);
}

constexpr int kObs = 128;  // observations per block in the gradient kernel
constexpr float kFixed = 1099511627776.0f;          // 2^40: resolution of the fixed-point sums
constexpr float kFixedMax = 4.611686018427388e18f;  // 2^62

// acc[i] += v * 2^40 rounded to an integer (two's complement in 64 bits,
// exact and associative); a non-finite v, or |v| >= 2^22 (a block's share of
// a mean gradient: only a diverged run gets there), is counted in
// acc[SM_CONF_PARAMS + 1] instead.
__device__ __forceinline__ void add_fixed(unsigned long long *acc, int i, float v)
{
    const float x = v * kFixed;
    if (fabsf(x) < kFixedMax)
        atomicAdd(acc + i, (unsigned long long)__float2ll_rn(x));
    else
        atomicAdd(acc + SM_CONF_PARAMS + 1, 1ull);
}

__device__ __forceinline__ float from_fixed(unsigned long long a)
{
    return (float)((double)(long long)a * (1.0 / 1099511627776.0));
}
// per-observation vectors kept for the block's reduction: x, h1, d_z1, h2, d_z2, d_o
constexpr int kRow = kF + 4 * kH + 1;

__global__ void __launch_bounds__(kObs)
    k_conf_grad(const float *__restrict__ params, const float *__restrict__ feat, const float *__restrict__ target,
                int64_t n, const int64_t *__restrict__ idx, int64_t n_obs, unsigned long long *__restrict__ acc)
{
    extern __shared__ float sm[];
    float *s = sm;                          // SM_CONF_PARAMS (bf16-rounded)
    float *rows = sm + SM_CONF_PARAMS + 3;  // kObs x kRow
    load_params(params, s);
    const int64_t i = (int64_t)blockIdx.x * kObs + threadIdx.x;
    float *r = rows + threadIdx.x * kRow;
    float l = 0.0f;
    // the minibatch's i-th observation: i itself, or idx[i] (an index outside
    // [0, n_obs) counts as a non-finite partial sum: the step's gradient and
    // loss become NaN, and the observation is not read)
    int64_t j = i;
    bool valid = i < n;
    if (valid && idx) {
        j = idx[i];
        if (j < 0 || j >= n_obs) {
            atomicAdd(acc + SM_CONF_PARAMS + 1, 1ull);
            valid = false;
        }
    }
    if (valid) {
        float x[kF], z1[kH], z2[kH];
#pragma unroll
        for (int k = 0; k < kF; ++k) x[k] = feat[j * kF + k];
        const float o = mlp_forward(s, x, z1, z2);
        const float y = target[j];
        l = (fmaxf(o, 0.0f) + log1pf(expf(-fabsf(o))) - y * o) / (float)n;  // softplus(o) - y o
        const float d_o = (1.0f / (1.0f + expf(-o)) - y) / (float)n;
        for (int k = 0; k < kF; ++k) r[k] = x[k];
        for (int j = 0; j < kH; ++j) {
            r[kF + 2 * kH + j] = fmaxf(z2[j], 0.0f);                          // h2
            r[kF + 3 * kH + j] = z2[j] > 0.0f ? d_o * s[kW3 + j] : 0.0f;      // d_z2
        }
        for (int a = 0; a < kH; ++a) {
            float acc = 0.0f;
            for (int j = 0; j < kH; ++j) acc = fmaf(r[kF + 3 * kH + j], s[kW2 + j * kH + a], acc);
            r[kF + a] = fmaxf(z1[a], 0.0f);                  // h1
            r[kF + kH + a] = z1[a] > 0.0f ? acc : 0.0f;      // d_z1
        }
        r[kF + 4 * kH] = d_o;
    } else {
        for (int k = 0; k < kRow; ++k) r[k] = 0.0f;
    }
    // block sum of the loss
    for (int off = 16; off > 0; off >>= 1) l += __shfl_xor_sync(0xffffffffu, l, off);
    if ((threadIdx.x & 31) == 0) add_fixed(acc, SM_CONF_PARAMS, l);
    __syncthreads();
    // each thread sums some parameters' gradients over the block's observations
    for (int q = threadIdx.x; q < SM_CONF_PARAMS; q += blockDim.x) {
        float g = 0.0f;
        for (int t = 0; t < kObs; ++t) {
            const float *rt = rows + t * kRow;
            float v;
            if (q < kB1) v = rt[kF + kH + q / kF] * rt[q % kF];                              // W1: d_z1 x
            else if (q < kW2) v = rt[kF + kH + (q - kB1)];                                    // b1
            else if (q < kB2) v = rt[kF + 3 * kH + (q - kW2) / kH] * rt[kF + (q - kW2) % kH];  // W2: d_z2 h1
            else if (q < kW3) v = rt[kF + 3 * kH + (q - kB2)];                                // b2
            else if (q < kB3) v = rt[kF + 4 * kH] * rt[kF + 2 * kH + (q - kW3)];              // w3: d_o h2
            else v = rt[kF + 4 * kH];                                                          // b3
            g += v;
        }
        add_fixed(acc, q, g);
    }
}

// acc: SM_CONF_PARAMS gradient sums, the loss, a count of non-finite partial
// sums; converts them to float32 (NaN everywhere once a partial sum was not
// finite) and takes the step.
__global__ void k_conf_update(float *__restrict__ params, const unsigned long long *__restrict__ acc, float lr,
                              float *__restrict__ grad, float *__restrict__ loss)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    const bool bad = acc[SM_CONF_PARAMS + 1] != 0ull;
    if (q < SM_CONF_PARAMS) {
        const float g = bad ? __int_as_float(0x7fc00000) : from_fixed(acc[q]);
        grad[q] = g;
        params[q] -= lr * g;
    } else if (q == SM_CONF_PARAMS) {
        *loss = bad ? __int_as_float(0x7fc00000) : from_fixed(acc[q]);
    }
}

__global__ void __launch_bounds__(256)
    k_conf_targets(const void *__restrict__ probs, sm_dtype dt, const float *__restrict__ scale, int c,
                   const int32_t *__restrict__ rows, int64_t n, const uint8_t *__restrict__ labels8, int64_t n_x,
                   float *__restrict__ y)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int32_t row = rows[p];
    float t = 0.0f;
    if (row >= 0 && row < n_x) {
        const float sc = (dt == SM_F32) ? 1.0f : scale[p];
        float m = -INFINITY;
        int am = 0;
        for (int j = 0; j < c; ++j) {
            const float v = load_p(probs, dt, p * c + j, sc);
            if (v > m) {
                m = v;
                am = j;
            }
        }
        t = (labels8[row] != 255 && am == labels8[row]) ? 1.0f : 0.0f;
    }
    y[p] = t;
}

}  // namespace

void launch_conf_features(const unsigned long long *keys, int64_t total, int H, int W, const float4 *V,
                          const int4 *faces, int64_t F, const sm_intrinsics *K, const double *T, const void *probs,
                          sm_dtype dt, const float *scale, int c, float *feat, cudaStream_t s)
{
    if (total <= 0) return;
    k_conf_features<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(keys, total, H, W, V, faces, F, K, T, probs, dt,
                                                                    scale, c, feat);
}

void launch_conf_weights(unsigned long long *keys, int64_t total, int H, int W, const float4 *V, const int4 *faces,
                         int64_t F, const sm_intrinsics *K, const double *T, const void *probs, sm_dtype dt,
                         const float *scale, int c, const float *params, float *w, int32_t *rows, cudaStream_t s)
{
    if (total <= 0) return;
    int64_t blocks = (total + 255) / 256;
    if (blocks > 8192) blocks = 8192;
    k_conf_weights<<<(unsigned)blocks, 256, 0, s>>>(keys, total, H, W, V, faces, F, K, T, probs, dt, scale, c, params,
                                                    w, rows);
}

void launch_conf_forward(const float *params, const float *feat, int64_t n, float *w, cudaStream_t s)
{
    if (n <= 0) return;
    k_conf_forward<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(params, feat, n, w);
}

cudaError_t launch_conf_train_step(float *params, const float *feat, const float *target, int64_t n, float lr,
                                   float *grad, float *loss, cudaStream_t s, const int64_t *idx, int64_t n_obs)
{
    // fixed-point sums: SM_CONF_PARAMS gradients, the loss, the non-finite count
    constexpr size_t kAccBytes = (SM_CONF_PARAMS + 2) * sizeof(unsigned long long);
    unsigned long long *acc = nullptr;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&acc), kAccBytes, s);
    if (e != cudaSuccess) return e;
    cudaMemsetAsync(acc, 0, kAccBytes, s);
    if (n > 0) {
        const size_t smem = (SM_CONF_PARAMS + 3 + (size_t)kObs * kRow) * sizeof(float);
        static PerDeviceOnce configured;
        if (configured.first(current_device()))
            cudaFuncSetAttribute(k_conf_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_conf_grad<<<(unsigned)((n + kObs - 1) / kObs), kObs, smem, s>>>(params, feat, target, n, idx, n_obs, acc);
    }
    k_conf_update<<<(SM_CONF_PARAMS + 1 + 255) / 256, 256, 0, s>>>(params, acc, lr, grad, loss);
    e = cudaGetLastError();
    const cudaError_t ef = cudaFreeAsync(acc, s);
    return e != cudaSuccess ? e : ef;
}

void launch_conf_targets(const void *probs, sm_dtype dt, const float *scale, int c, const int32_t *rows, int64_t n,
                         const uint8_t *labels8, int64_t n_x, float *y, cudaStream_t s)
{
    if (n <= 0) return;
    k_conf_targets<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(probs, dt, scale, c, rows, n, labels8, n_x, y);
}

}  // namespace lf
