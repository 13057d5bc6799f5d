// Aggregator kernels (Sec. 3.2, 3.3.2): per-frame row histogram for the image
// weights w^(I) = 1/|K_i ∩ K_x| (Sec. 3.2.2), the scatter of every pixel's
// probability vector into its row of the accumulator array P (Eq.
// texel-in-array) under the fusion rules (Eqs. sum, mul, maxsum and their
// weighted forms), normalisation + arg max (Sec. 3.2.1) and render-back.
#include <cuda_bf16.h>

#include "lf_internal.cuh"

namespace lf {
namespace {

// Decoders of the stored probability types.  E4M3 (1 sign, 4 exponent bits
// with bias 7, 3 mantissa bits, no infinities, S.1111.111 = NaN) is decoded
// from its definition: subnormals m * 2^-9, normals (1 + m/8) 2^(e-7).
__device__ __forceinline__ float decode_e4m3(uint8_t b)
{
    const uint32_t s = b >> 7, e = (b >> 3) & 0xF, m = b & 7;
    float v;
    if (e == 0) {
        v = (float)m * 0.001953125f;  // 2^-9
    } else if (e == 15 && m == 7) {
        v = __int_as_float(0x7fc00000);
    } else {
        v = __uint_as_float(((e + 120u) << 23) | (m << 20));
    }
    return s ? -v : v;
}

template <int DT>
__device__ __forceinline__ float load_prob(const void *base, int64_t idx)
{
    if (DT == SM_F32) return __ldcs(reinterpret_cast<const float *>(base) + idx);
    if (DT == SM_BF16) {
        const unsigned short q = __ldcs(reinterpret_cast<const unsigned short *>(base) + idx);
        return __uint_as_float((uint32_t)q << 16);
    }
    const uint8_t q = reinterpret_cast<const uint8_t *>(base)[idx];
    return decode_e4m3(q);
}

// |K_i ∩ K_x| for every frame i of the batch and row x: histogram of the row
// map, or of the z-buffer keys (face mode, row = triangle) when idmap is null.
// kPixUnroll pixels per thread (see kPixThreads); the pixels of one run of a
// row within a warp add their count with one atomic.
__global__ void __launch_bounds__(kPixThreads) k_count(const int32_t *__restrict__ idmap,
                                                       const unsigned long long *__restrict__ keys, int64_t total,
                                                       int64_t npix, uint32_t *__restrict__ fcnt, int64_t n_x)
{
    const int64_t base = (int64_t)blockIdx.x * kPixPerBlock;
    const int lane = threadIdx.x & 31;
    int32_t row[kPixUnroll];
#pragma unroll
    for (int j = 0; j < kPixUnroll; ++j) {
        const int64_t p = base + j * kPixThreads + threadIdx.x;
        row[j] = -1;
        if (p < total) {
            if (idmap) {
                row[j] = idmap[p];
            } else {
                const unsigned long long key = keys[p];
                row[j] = (key == kEmptyKey) ? -1 : (int32_t)(unsigned int)key;
            }
        }
    }
    FrameCursor fc(base, npix);
#pragma unroll
    for (int j = 0; j < kPixUnroll; ++j) {
        const int64_t p = base + j * kPixThreads + threadIdx.x;
        const int64_t f = fc.at(p < total ? p : total - 1);
        const int n = warp_run_length(((unsigned long long)f << 32) | (unsigned int)row[j], lane);
        if (n && row[j] >= 0 && row[j] < n_x) atomicAdd(fcnt + f * n_x + row[j], (uint32_t)n);
    }
}

__global__ void __launch_bounds__(kPixThreads) k_count_reset(const int32_t *__restrict__ idmap, int64_t total,
                                                             int64_t npix, uint32_t *__restrict__ fcnt, int64_t n_x)
{
    const int64_t base = (int64_t)blockIdx.x * kPixPerBlock;
    const int lane = threadIdx.x & 31;
    int32_t row[kPixUnroll];
#pragma unroll
    for (int j = 0; j < kPixUnroll; ++j) {
        const int64_t p = base + j * kPixThreads + threadIdx.x;
        row[j] = p < total ? idmap[p] : -1;
    }
    FrameCursor fc(base, npix);
#pragma unroll
    for (int j = 0; j < kPixUnroll; ++j) {
        const int64_t p = base + j * kPixThreads + threadIdx.x;
        const int64_t f = fc.at(p < total ? p : total - 1);
        const int n = warp_run_length(((unsigned long long)f << 32) | (unsigned int)row[j], lane);
        if (n && row[j] >= 0 && row[j] < n_x) fcnt[f * n_x + row[j]] = 0u;
    }
}

// Visible-area pre-pass of the texel steps (Sec. 3.1; a_t read as the most
// pixels a triangle is visible on in one frame).  kPixUnroll pixels of a
// batch's z-buffers per thread: the winning triangle's per-frame count grows
// by its pixels (one atomic per run within a warp), and the key is re-armed
// for the next batch.
__global__ void __launch_bounds__(kPixThreads) k_area_count(unsigned long long *__restrict__ keys, int64_t total,
                                                            int64_t npix, uint32_t *__restrict__ fcnt, int64_t F)
{
    const int64_t base = (int64_t)blockIdx.x * kPixPerBlock;
    const int lane = threadIdx.x & 31;
    unsigned long long key[kPixUnroll];
#pragma unroll
    for (int j = 0; j < kPixUnroll; ++j) {
        const int64_t p = base + j * kPixThreads + threadIdx.x;
        key[j] = p < total ? keys[p] : kEmptyKey;
    }
    FrameCursor fc(base, npix);
#pragma unroll
    for (int j = 0; j < kPixUnroll; ++j) {
        const int64_t p = base + j * kPixThreads + threadIdx.x;
        if (key[j] != kEmptyKey) keys[p] = kEmptyKey;
        const int64_t f = fc.at(p < total ? p : total - 1);
        const int32_t t = key[j] == kEmptyKey ? -1 : (int32_t)(unsigned int)key[j];
        const int n = warp_run_length(((unsigned long long)f << 32) | (unsigned int)t, lane);
        if (n && t >= 0 && t < F) atomicAdd(fcnt + f * F + t, (uint32_t)n);
    }
}

// One thread per triangle: the largest of its nb per-frame counts folded into
// area[f]; the counts are zeroed for the next batch.
__global__ void k_area_max(uint32_t *__restrict__ fcnt, int nb, int64_t F, int32_t *__restrict__ area)
{
    const int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= F) return;
    uint32_t m = (uint32_t)area[f];
    for (int b = 0; b < nb; ++b) {
        const uint32_t v = fcnt[(int64_t)b * F + f];
        if (v) {
            m = v > m ? v : m;
            fcnt[(int64_t)b * F + f] = 0u;
        }
    }
    area[f] = (int32_t)m;
}

// s_t = max(1, ceil(gamma sqrt(a_t))) in binary32 with correctly rounded
// square root and product (Sec. 3.1).
__global__ void k_texel_res(const int32_t *__restrict__ area, int64_t F, float gamma, int32_t *__restrict__ s_out)
{
    const int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= F) return;
    const float c = ceilf(__fmul_rn(gamma, __fsqrt_rn((float)area[f])));
    s_out[f] = c < 1.0f ? 1 : (int32_t)c;
}

// One thread per pixel: phi(p) of the pixel's prediction, times its weight,
// added into its row with float atomics; the row's observation count + 1.
//   sum    phi = p
//   logsum phi = log(max(p, 2^-30))   (Eq. mul as a sum of logarithms)
//   maxsum phi = g(p): entries equal to max p keep their value, others 0
//   vote   phi = onehot(first arg max p)
template <int RULE, int DT>
__global__ void __launch_bounds__(256)
    k_scatter(const void *__restrict__ probs, const float *__restrict__ scale, const int32_t *__restrict__ idmap,
              int64_t total, int64_t npix, int c, const uint32_t *__restrict__ fcnt, float alpha,
              const float *__restrict__ wpix, int64_t n_x,
              float *__restrict__ acc, uint32_t *__restrict__ cnt, int32_t *__restrict__ err)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= total) return;
    const int32_t row = idmap[p];
    if (row < 0) return;
    if (row >= n_x) {
        atomicCAS(err, 0, (int32_t)kErrRowRange);
        return;
    }
    float w = 1.0f;
    if (wpix) w = wpix[p];
    else if (fcnt) w = image_weight(alpha, fcnt[frame_of(p, npix) * n_x + row]);
    const float sc = (DT == SM_F32) ? 1.0f : scale[p];
    float *a = acc + (int64_t)row * c;
    const int64_t base = p * c;
    if (RULE == SM_RULE_SUM || RULE == SM_RULE_LOGSUM) {
        for (int j = 0; j < c; ++j) {
            float v = load_prob<DT>(probs, base + j);
            if (DT != SM_F32) v = __fmul_rn(v, sc);
            const float phi = (RULE == SM_RULE_SUM) ? v : logf(fmaxf(v, kPMin));
            atomicAdd(a + j, __fmul_rn(w, phi));
        }
    } else {
        float m = -INFINITY;
        int am = 0;
        for (int j = 0; j < c; ++j) {
            float v = load_prob<DT>(probs, base + j);
            if (DT != SM_F32) v = __fmul_rn(v, sc);
            if (j == 0 || v > m) {
                m = v;
                am = j;
            }
        }
        if (RULE == SM_RULE_VOTE) {
            atomicAdd(a + am, w);
        } else {
            for (int j = 0; j < c; ++j) {
                float v = load_prob<DT>(probs, base + j);
                if (DT != SM_F32) v = __fmul_rn(v, sc);
                if (v == m) atomicAdd(a + j, __fmul_rn(w, v));
            }
        }
    }
    atomicAdd(cnt + row, 1u);
}

// One thread per row: label = first arg max of the accumulator; distribution
// L1-normalised (sum/maxsum/vote) or exp(L - max L) / sum exp(L - max L)
// (logsum).  Unobserved rows: label -1 (255 in the uint8 copy), zero row.
__global__ void k_normalise(int rule, const float *__restrict__ acc, const uint32_t *__restrict__ cnt, int64_t n_x,
                            int c, float *__restrict__ dist, int32_t *__restrict__ labels,
                            uint8_t *__restrict__ labels8)
{
    const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= n_x) return;
    const float *a = acc + l * c;
    if (cnt[l] == 0) {
        labels8[l] = 255;
        if (labels) labels[l] = -1;
        if (dist)
            for (int j = 0; j < c; ++j) dist[l * c + j] = 0.0f;
        return;
    }
    int am = 0;
    float m = a[0];
    for (int j = 1; j < c; ++j) {
        const float v = a[j];
        if (v > m) {
            m = v;
            am = j;
        }
    }
    labels8[l] = (uint8_t)am;
    if (labels) labels[l] = am;
    if (!dist) return;
    float total = 0.0f;
    if (rule == SM_RULE_LOGSUM) {
        for (int j = 0; j < c; ++j) total += expf(a[j] - m);
        const float inv = 1.0f / total;
        for (int j = 0; j < c; ++j) dist[l * c + j] = expf(a[j] - m) * inv;
    } else {
        for (int j = 0; j < c; ++j) total += a[j];
        const float inv = 1.0f / total;
        for (int j = 0; j < c; ++j) dist[l * c + j] = a[j] * inv;
    }
}

__global__ void k_render(const int32_t *__restrict__ idmap, int64_t npix, const uint8_t *__restrict__ labels8,
                         int64_t n_x, uint8_t *__restrict__ out)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npix) return;
    const int32_t row = idmap[p];
    out[p] = (row < 0 || row >= n_x) ? (uint8_t)255 : labels8[row];
}

// 16 pixels per thread: four 16-byte row-map loads, one 16-byte label store;
// a pixel on the same row as the previous one reuses its label (runs of a
// few pixels per triangle are the rule), so most label gathers are skipped.
__global__ void k_render16(const int4 *__restrict__ idmap, int64_t n16, const uint8_t *__restrict__ labels8,
                           int64_t n_x, uint4 *__restrict__ out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n16) return;
    int4 r[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) r[j] = __ldcs(idmap + 4 * i + j);
    uint32_t w[4];
    int prev = -1;
    uint32_t plab = 255u;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int rr[4] = {r[j].x, r[j].y, r[j].z, r[j].w};
        uint32_t packed = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (rr[k] != prev) {
                plab = (rr[k] < 0 || rr[k] >= n_x) ? 255u : (uint32_t)labels8[rr[k]];
                prev = rr[k];
            }
            packed |= plab << (8 * k);
        }
        w[j] = packed;
    }
    __stcs(out + i, make_uint4(w[0], w[1], w[2], w[3]));
}

template <int RULE>
void scatter_dt(sm_dtype dt, dim3 g, cudaStream_t s, const void *probs, const float *scale, const int32_t *idmap,
                int64_t total, int64_t npix, int c, const uint32_t *fcnt, float alpha, const float *wpix, int64_t n_x, float *acc,
                uint32_t *cnt, int32_t *err)
{
    if (dt == SM_F32)
        k_scatter<RULE, SM_F32>
            <<<g, 256, 0, s>>>(probs, scale, idmap, total, npix, c, fcnt, alpha, wpix, n_x, acc, cnt, err);
    else if (dt == SM_BF16)
        k_scatter<RULE, SM_BF16>
            <<<g, 256, 0, s>>>(probs, scale, idmap, total, npix, c, fcnt, alpha, wpix, n_x, acc, cnt, err);
    else
        k_scatter<RULE, SM_FP8_E4M3>
            <<<g, 256, 0, s>>>(probs, scale, idmap, total, npix, c, fcnt, alpha, wpix, n_x, acc, cnt, err);
}

}  // namespace

void launch_count(const int32_t *idmap, const unsigned long long *keys, int64_t npix, int nb, uint32_t *fcnt,
                  int64_t n_x, cudaStream_t s)
{
    const int64_t total = npix * nb;
    if (total <= 0) return;
    k_count<<<(unsigned)((total + kPixPerBlock - 1) / kPixPerBlock), kPixThreads, 0, s>>>(idmap, keys, total, npix,
                                                                                           fcnt, n_x);
}

void launch_area_count(unsigned long long *keys, int64_t npix, int nb, uint32_t *fcnt, int64_t F, cudaStream_t s)
{
    const int64_t total = npix * nb;
    if (total <= 0) return;
    k_area_count<<<(unsigned)((total + kPixPerBlock - 1) / kPixPerBlock), kPixThreads, 0, s>>>(keys, total, npix,
                                                                                                fcnt, F);
}

void launch_area_max(uint32_t *fcnt, int nb, int64_t F, int32_t *area, cudaStream_t s)
{
    if (F <= 0 || nb <= 0) return;
    k_area_max<<<(unsigned)((F + 255) / 256), 256, 0, s>>>(fcnt, nb, F, area);
}

void launch_texel_res(const int32_t *area, int64_t F, float gamma, int32_t *s_out, cudaStream_t s)
{
    if (F <= 0) return;
    k_texel_res<<<(unsigned)((F + 255) / 256), 256, 0, s>>>(area, F, gamma, s_out);
}

void launch_count_reset(const int32_t *idmap, int64_t npix, int nb, uint32_t *fcnt, int64_t n_x, cudaStream_t s)
{
    const int64_t total = npix * nb;
    if (total <= 0) return;
    k_count_reset<<<(unsigned)((total + kPixPerBlock - 1) / kPixPerBlock), kPixThreads, 0, s>>>(idmap, total, npix,
                                                                                                 fcnt, n_x);
}

void launch_scatter(sm_rule rule, sm_dtype dtype, const void *probs, const float *scale, const int32_t *idmap,
                    int64_t npix, int nb, int c, const uint32_t *fcnt, float alpha, const float *wpix, int64_t n_x, float *acc,
                    uint32_t *cnt, int32_t *err, cudaStream_t s)
{
    const int64_t total = npix * nb;
    if (total <= 0) return;
    dim3 g((unsigned)((total + 255) / 256));
    switch (rule) {
    case SM_RULE_SUM:
        scatter_dt<SM_RULE_SUM>(dtype, g, s, probs, scale, idmap, total, npix, c, fcnt, alpha, wpix, n_x, acc, cnt, err);
        break;
    case SM_RULE_LOGSUM:
        scatter_dt<SM_RULE_LOGSUM>(dtype, g, s, probs, scale, idmap, total, npix, c, fcnt, alpha, wpix, n_x, acc, cnt, err);
        break;
    case SM_RULE_MAXSUM:
        scatter_dt<SM_RULE_MAXSUM>(dtype, g, s, probs, scale, idmap, total, npix, c, fcnt, alpha, wpix, n_x, acc, cnt, err);
        break;
    default:
        scatter_dt<SM_RULE_VOTE>(dtype, g, s, probs, scale, idmap, total, npix, c, fcnt, alpha, wpix, n_x, acc, cnt, err);
        break;
    }
}

void launch_normalise(sm_rule rule, const float *acc, const uint32_t *cnt, int64_t n_x, int c, float *dist,
                      int32_t *labels, uint8_t *labels8, cudaStream_t s)
{
    if (n_x <= 0) return;
    k_normalise<<<(unsigned)((n_x + 255) / 256), 256, 0, s>>>((int)rule, acc, cnt, n_x, c, dist, labels, labels8);
}

void launch_render(const int32_t *idmap, int64_t npix, const uint8_t *labels8, int64_t n_x, uint8_t *out,
                   cudaStream_t s)
{
    if (npix <= 0) return;
    int64_t done = 0;
    if (((uintptr_t)idmap & 15) == 0 && ((uintptr_t)out & 15) == 0) {
        const int64_t n16 = npix / 16;
        if (n16 > 0)
            k_render16<<<(unsigned)((n16 + 255) / 256), 256, 0, s>>>(reinterpret_cast<const int4 *>(idmap), n16,
                                                                      labels8, n_x, reinterpret_cast<uint4 *>(out));
        done = n16 * 16;
    }
    if (done < npix)
        k_render<<<(unsigned)((npix - done + 255) / 256), 256, 0, s>>>(idmap + done, npix - done, labels8, n_x,
                                                                        out + done);
}

}  // namespace lf
