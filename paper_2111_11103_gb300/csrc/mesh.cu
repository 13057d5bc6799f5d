// Mesh upload kernels (Sec. 3.1, 3.3.2): vertex/face packing with index
// validation, per-triangle texel layout (texel steps s, uv origin) and the
// exclusive prefix sum of the texel counts that gives every triangle its
// first row id_t.
#include "lf_internal.cuh"

namespace lf {
namespace {

constexpr int kScanBlock = 1024;  // threads per scan block
constexpr int kScanItems = 4;     // elements per thread
constexpr int kScanTile = kScanBlock * kScanItems;

__global__ void k_pack(const float *__restrict__ verts, int64_t V, const int32_t *__restrict__ faces, int64_t F,
                       float4 *__restrict__ v4, int4 *__restrict__ f4, int32_t *__restrict__ err)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < V) v4[i] = make_float4(verts[3 * i], verts[3 * i + 1], verts[3 * i + 2], 0.0f);
    if (i < F) {
        const int a = faces[3 * i], b = faces[3 * i + 1], c = faces[3 * i + 2];
        const bool ok = a >= 0 && a < V && b >= 0 && b < V && c >= 0 && c < V;
        if (!ok) atomicCAS(err, 0, (int32_t)kErrFaceIndex);
        f4[i] = make_int4(ok ? a : 0, ok ? b : 0, ok ? c : 0, ok ? 1 : 0);
    }
}

// uv origin (Sec. 3.1): the vertex whose interior angle is closest to 90
// degrees, i.e. the smallest cos^2 = dot^2 / (|e1|^2 |e2|^2); lowest local index
// on ties; binary32 with explicit rounding (the choice is an integer).
__device__ int uv_origin(float4 p0, float4 p1, float4 p2)
{
    const float4 p[3] = {p0, p1, p2};
    float best = 0.0f;
    int best_k = 0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float4 a = p[k], b = p[(k + 1) % 3], c = p[(k + 2) % 3];
        const float e1x = __fsub_rn(b.x, a.x), e1y = __fsub_rn(b.y, a.y), e1z = __fsub_rn(b.z, a.z);
        const float e2x = __fsub_rn(c.x, a.x), e2y = __fsub_rn(c.y, a.y), e2z = __fsub_rn(c.z, a.z);
        const float dot = __fadd_rn(__fadd_rn(__fmul_rn(e1x, e2x), __fmul_rn(e1y, e2y)), __fmul_rn(e1z, e2z));
        const float n1 = __fadd_rn(__fadd_rn(__fmul_rn(e1x, e1x), __fmul_rn(e1y, e1y)), __fmul_rn(e1z, e1z));
        const float n2 = __fadd_rn(__fadd_rn(__fmul_rn(e2x, e2x), __fmul_rn(e2y, e2y)), __fmul_rn(e2z, e2z));
        const float den = __fmul_rn(n1, n2);
        const float q = (den > 0.0f) ? __fdiv_rn(__fmul_rn(dot, dot), den) : 2.0f;
        if (k == 0 || q < best) {
            best = q;
            best_k = k;
        }
    }
    return best_k;
}

__device__ __forceinline__ int64_t texel_count(int s) { return ((int64_t)s * s + s) / 2; }

// Per triangle: validated s, uv origin, texel count; per block: the block's
// total (first pass of the scan).
__global__ void __launch_bounds__(kScanBlock)
    k_texel_info(const int32_t *__restrict__ res, const float4 *__restrict__ v4, const int4 *__restrict__ f4,
                 int64_t F, int32_t *__restrict__ texinfo, int64_t *__restrict__ block_sums,
                 int32_t *__restrict__ err)
{
    __shared__ int64_t red[kScanBlock / 32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    int64_t local = 0;
#pragma unroll
    for (int it = 0; it < kScanItems; ++it) {
        const int64_t f = base + (int64_t)it * kScanBlock + threadIdx.x;
        if (f >= F) continue;
        int s = res[f];
        if (s < 1 || s > SM_MAX_TEXEL_RES) {
            atomicCAS(err, 0, (int32_t)kErrTexelRes);
            s = 1;
        }
        int o = 0;
        if (s > 1) {
            const int4 fc = f4[f];
            o = uv_origin(v4[fc.x], v4[fc.y], v4[fc.z]);
        }
        texinfo[f] = s | (o << 16);
        local += texel_count(s);
    }
    for (int off = 16; off > 0; off >>= 1) local += __shfl_down_sync(0xffffffffu, local, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = local;
    __syncthreads();
    if (threadIdx.x < 32) {
        int64_t v = red[threadIdx.x];
        for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
        if (threadIdx.x == 0) block_sums[blockIdx.x] = v;
    }
}

// Exclusive scan of the block totals by a single block (sequential chunks per
// thread, then a block-wide scan of the chunk sums); writes n_x.
__global__ void __launch_bounds__(kScanBlock)
    k_scan_blocks(int64_t *__restrict__ block_sums, int64_t nblocks, int64_t *__restrict__ n_x_out,
                  int32_t *__restrict__ err)
{
    __shared__ int64_t sh[kScanBlock];
    const int64_t per = (nblocks + kScanBlock - 1) / kScanBlock;
    const int64_t lo = threadIdx.x * per, hi = min(lo + per, nblocks);
    int64_t sum = 0;
    for (int64_t i = lo; i < hi; ++i) sum += block_sums[i];
    sh[threadIdx.x] = sum;
    __syncthreads();
    for (int off = 1; off < kScanBlock; off <<= 1) {  // Hillis-Steele inclusive scan
        int64_t v = (threadIdx.x >= off) ? sh[threadIdx.x - off] : 0;
        __syncthreads();
        sh[threadIdx.x] += v;
        __syncthreads();
    }
    int64_t run = sh[threadIdx.x] - sum;  // exclusive prefix of this thread's chunk
    for (int64_t i = lo; i < hi; ++i) {
        const int64_t v = block_sums[i];
        block_sums[i] = run;
        run += v;
    }
    if (threadIdx.x == kScanBlock - 1) {
        *n_x_out = sh[kScanBlock - 1];
        if (sh[kScanBlock - 1] >= 2147483647LL) atomicCAS(err, 0, (int32_t)kErrRowOverflow);
    }
}

// Block-local exclusive scan of the texel counts plus the block offset.
__global__ void __launch_bounds__(kScanBlock)
    k_scan_apply(const int32_t *__restrict__ texinfo, int64_t F, const int64_t *__restrict__ block_offsets,
                 int32_t *__restrict__ row0)
{
    __shared__ int64_t warp_tot[kScanBlock / 32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int64_t v[kScanItems];
    int64_t mine = 0;
#pragma unroll
    for (int it = 0; it < kScanItems; ++it) {
        const int64_t f = base + it;
        v[it] = (f < F) ? texel_count(texinfo[f] & 0xFFFF) : 0;
        mine += v[it];
    }
    // warp inclusive scan of per-thread sums
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t inc = mine;
    for (int off = 1; off < 32; off <<= 1) {
        const int64_t t = __shfl_up_sync(0xffffffffu, inc, off);
        if (lane >= off) inc += t;
    }
    if (lane == 31) warp_tot[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        int64_t w = warp_tot[lane];
        for (int off = 1; off < 32; off <<= 1) {
            const int64_t t = __shfl_up_sync(0xffffffffu, w, off);
            if (lane >= off) w += t;
        }
        warp_tot[lane] = w;  // inclusive over warps
    }
    __syncthreads();
    int64_t run = block_offsets[blockIdx.x] + (warp > 0 ? warp_tot[warp - 1] : 0) + inc - mine;
#pragma unroll
    for (int it = 0; it < kScanItems; ++it) {
        const int64_t f = base + it;
        if (f < F) row0[f] = (int32_t)run;
        run += v[it];
    }
}

}  // namespace

void launch_pack_mesh(const float *verts, int64_t V, const int32_t *faces, int64_t F, float4 *verts4, int4 *faces4,
                      int32_t *err, cudaStream_t s)
{
    const int64_t n = V > F ? V : F;
    if (n <= 0) return;
    k_pack<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(verts, V, faces, F, verts4, faces4, err);
}

size_t texel_scan_scratch_bytes(int64_t F)
{
    const int64_t nblocks = (F + kScanTile - 1) / kScanTile;
    return (size_t)(nblocks > 0 ? nblocks : 1) * sizeof(int64_t);
}

void launch_texel_layout(const int32_t *res, const float4 *verts4, const int4 *faces4, int64_t F, int32_t *texinfo,
                         int32_t *row0, int64_t *n_x_out, void *scratch, int32_t *err, cudaStream_t s)
{
    const int64_t nblocks = (F + kScanTile - 1) / kScanTile;
    int64_t *block_sums = static_cast<int64_t *>(scratch);
    if (nblocks <= 0) {
        cudaMemsetAsync(n_x_out, 0, sizeof(int64_t), s);
        return;
    }
    k_texel_info<<<(unsigned)nblocks, kScanBlock, 0, s>>>(res, verts4, faces4, F, texinfo, block_sums, err);
    k_scan_blocks<<<1, kScanBlock, 0, s>>>(block_sums, nblocks, n_x_out, err);
    k_scan_apply<<<(unsigned)nblocks, kScanBlock, 0, s>>>(texinfo, F, block_sums, row0);
}

}  // namespace lf
