// Internal declarations shared by the library's translation units.
#pragma once

#include <atomic>

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "labelfuse.h"

namespace lf {

// Per-frame camera: rows 0/1 map a world point to (image x, image y) * Z in
// 1/256-pixel units, row 2 to the camera depth Z (all binary32).
struct Camera {
    float a[12];
};

constexpr float kZNear = 0.05f;             // a vertex at depth <= this drops its triangle
constexpr float kSnapLimit = 536870912.0f;  // |snapped coordinate| <= 2^29 (int64 edge products stay exact)
constexpr float kPMin = 9.31322574615478515625e-10f;  // 2^-30, lower clamp before log
constexpr unsigned long long kEmptyKey = ~0ull;

// Per-pixel kernels over a batch of frames (resolve, row histograms): a block
// of kPixThreads threads takes kPixUnroll * kPixThreads consecutive pixels,
// thread t the pixels base + j * kPixThreads + t (j < kPixUnroll), so every
// load is one coalesced warp access and kPixUnroll of them are in flight per
// thread before any result is used (one load per thread leaves a memory-bound
// kernel far below the HBM bandwidth).
constexpr int kPixThreads = 256;
constexpr int kPixUnroll = 8;
constexpr int64_t kPixPerBlock = (int64_t)kPixThreads * kPixUnroll;

#ifdef __CUDACC__
// Frame of pixel p of a batch: a 32-bit division where both fit (several
// times cheaper than the 64-bit one).
__device__ __forceinline__ int64_t frame_of(int64_t p, int64_t npix)
{
    if (((uint64_t)p | (uint64_t)npix) <= 0xffffffffull) return (int64_t)((uint32_t)p / (uint32_t)npix);
    return p / npix;
}

// Frame of pixel p for non-decreasing p (no division per pixel).
struct FrameCursor {
    int64_t f, end, npix;
    __device__ __forceinline__ FrameCursor(int64_t p, int64_t npix_) : f(p / npix_), end((p / npix_ + 1) * npix_), npix(npix_) {}
    __device__ __forceinline__ int64_t at(int64_t p)
    {
        while (p >= end) {
            ++f;
            end += npix;
        }
        return f;
    }
};

// Runs of equal keys over a warp's 32 lanes (lane = consecutive pixel): the
// length of the run that starts at this lane, 0 if the lane does not start
// one.  Every lane of the warp must call it.
__device__ __forceinline__ int warp_run_length(unsigned long long key, int lane)
{
    const unsigned long long prev = __shfl_up_sync(0xffffffffu, key, 1);
    const bool start = lane == 0 || key != prev;
    const unsigned int S = __ballot_sync(0xffffffffu, start);
    if (!start) return 0;
    const unsigned int above = lane == 31 ? 0u : S & ~((2u << lane) - 1u);
    return (above ? __ffs(above) - 1 : 32) - lane;
}
#endif

// Error codes latched by kernels (first one wins).
enum DeviceError : int32_t {
    kErrNone = 0,
    kErrFaceIndex = 1,    // a face references a vertex outside [0, V)
    kErrTexelRes = 2,     // texel steps outside [1, SM_MAX_TEXEL_RES]
    kErrRowRange = 3,     // a row index outside [0, n_x) reached the scatter
    kErrRowOverflow = 4,  // n_x >= 2^31
    kErrTimeout = 5,      // a bounded wait inside a kernel gave up
};

// ---- kernels (raster.cu) ----
void launch_project(const sm_intrinsics *K, const double *T, int N, Camera *out, cudaStream_t s);
// Faces are processed in clusters of 32 (one warp); bounds holds two float4
// (min, max corner; min.w != 0 marks a cluster without valid faces) per cluster.
constexpr int kClusterFaces = 32;

// Remembers, per device ordinal (< 64), that a per-device setting of a kernel
// (cudaFuncSetAttribute applies to the current device) has been made.
struct PerDeviceOnce {
    std::atomic<uint64_t> done{0};
    bool first(int dev)
    {
        const uint64_t bit = 1ull << (dev & 63);
        return !(done.fetch_or(bit) & bit);
    }
};
__host__ inline int current_device()
{
    int dev = 0;
    cudaGetDevice(&dev);
    return dev;
}

// Image weight of a pixel whose row holds n pixels of its frame, mixed with
// the pixel weight (Fig. 5a, read as a linear mix): (1 - alpha) + alpha / n in
// binary32; alpha = 1 gives w^(I) = 1/n exactly, alpha = 0 gives 1.
__device__ __forceinline__ float image_weight(float alpha, uint32_t n)
{
    return __fadd_rn(1.0f - alpha, __fmul_rn(alpha, __fdiv_rn(1.0f, (float)n)));
}
void launch_cluster_bounds(const float4 *V, const int4 *faces, int64_t F, float4 *bounds, cudaStream_t s);
// Raster of frames [frame0, frame0 + nb) into keys (nb x H x W z-buffer
// keys): a cluster cull pass writes per-frame lists of the clusters that may
// be visible (list: nb x ncl entries, count: nb), then the listed clusters
// are rasterised.
void launch_raster(const float4 *V, const int4 *faces, int64_t F, const float4 *bounds, const Camera *cams,
                   int frame0, int nb, int H, int W, unsigned long long *keys, int32_t *list, uint32_t *count,
                   cudaStream_t s);
void launch_resolve(unsigned long long *keys, int nb, int H, int W, const int32_t *row0, const int32_t *texinfo,
                    const float4 *V, const int4 *faces, const Camera *cams, int frame0, int32_t *idmap,
                    int32_t *idmap2, cudaStream_t s);

// Row maps of N frames with the library's static scratch (no allocation).
cudaError_t launch_render_rows_noalloc(const float *V, int64_t nV, const int32_t *faces, int64_t F,
                                       const sm_intrinsics *K, const double *T, int N, int H, int W, int32_t *idmap,
                                       cudaStream_t s);

// ---- kernels (fuse.cu) ----
// Row histogram from a row map, or (idmap == null) from z-buffer keys.
void launch_count(const int32_t *idmap, const unsigned long long *keys, int64_t npix, int nb, uint32_t *fcnt,
                  int64_t n_x, cudaStream_t s);
void launch_count_reset(const int32_t *idmap, int64_t npix, int nb, uint32_t *fcnt, int64_t n_x, cudaStream_t s);
void launch_scatter(sm_rule rule, sm_dtype dtype, const void *probs, const float *scale, const int32_t *idmap,
                    int64_t npix, int nb, int c, const uint32_t *fcnt, float alpha, const float *wpix, int64_t n_x,
                    float *acc, uint32_t *cnt, int32_t *err, cudaStream_t s);
// Pipelined scatter (scatter.cu): TMA-streamed tiles, run-length
// pre-reduction in registers, vector reductions into the rows.  Face mode
// passes the z-buffer keys (read, re-armed, optionally written out as row
// map); texel mode passes the resolved row map.  Requires
// scatter_tma_supported(c).
bool scatter_tma_supported(int c);
void launch_scatter_tma(sm_rule rule, sm_dtype dtype, const void *probs, const float *scale,
                        unsigned long long *keys, const int32_t *ids_in, int32_t *ids_out, int64_t total_px,
                        int64_t npix, int c, const uint32_t *fcnt, float alpha, const float *wpix, int64_t n_x,
                        float *acc, uint32_t *cnt, int32_t *err, cudaStream_t s);
// Persistent fusion kernel with a device work queue (queue.cu): raster and
// scatter of up to fuse_queue_max_scenes() scene pieces with at most
// fuse_queue_max_batches() batches in all, in one launch (face mode, pixel
// weights; one class count, 20 or 40, one storage type and one rule per
// launch; no two pieces of one mesh).  Per piece: nb batches of B frames
// into `slots` z-buffer slots of slot_stride keys (slots > lookahead), all
// keys empty on entry and on return.  counters: fuse_queue_counter_words(G)
// words for G batches in all, zeroed by the launch.
struct FuseQueueScene {
    const float4 *V;
    const int4 *faces;
    int64_t F;
    const float4 *bounds;
    const Camera *cams;  // first frame of the piece
    int H, W;
    int64_t npix;
    const void *probs;   // first frame of the piece
    const float *scale;
    int32_t *ids_out;    // optional, first frame of the piece
    float *acc;
    uint32_t *cnt;
    int64_t n_x;
    int32_t *err;
    unsigned long long *keys;
    int64_t slot_stride;
    int slots;
    int nb, B;
    int raster_rounds;   // cull rounds (fuse_queue_raster_round() clusters each) per raster item
    int scatter_tiles;   // 256-pixel tiles per scatter item
    const void *owner;   // the mesh the piece belongs to
};
bool fuse_queue_supported(int c);
int fuse_queue_raster_round();
int fuse_queue_max_scenes();
int fuse_queue_max_batches();
uint32_t fuse_queue_counter_words(int G);
// false (nothing enqueued) if the pieces break a limit above
bool launch_fuse_queue(const FuseQueueScene *scenes, int n, sm_dtype dtype, int c, sm_rule rule, int lookahead,
                       uint32_t *counters, cudaStream_t s);

// Visible-area pre-pass (fuse.cu): per-frame pixel counts of the triangles in
// a batch's z-buffers (re-armed), folded into per-triangle maxima; texel
// steps from the maxima.
void launch_area_count(unsigned long long *keys, int64_t npix, int nb, uint32_t *fcnt, int64_t F, cudaStream_t s);
void launch_area_max(uint32_t *fcnt, int nb, int64_t F, int32_t *area, cudaStream_t s);
void launch_texel_res(const int32_t *area, int64_t F, float gamma, int32_t *s_out, cudaStream_t s);
// Learned per-observation confidence (confidence.cu).
void launch_conf_features(const unsigned long long *keys, int64_t total, int H, int W, const float4 *V,
                          const int4 *faces, int64_t F, const sm_intrinsics *K, const double *T, const void *probs,
                          sm_dtype dt, const float *scale, int c, float *feat, cudaStream_t s);
void launch_conf_forward(const float *params, const float *feat, int64_t n, float *w, cudaStream_t s);
// Features and network output in one pass over a rasterised batch (tensor
// cores for the hidden layer); writes weights and the row map, re-arms keys.
void launch_conf_weights(unsigned long long *keys, int64_t total, int H, int W, const float4 *V, const int4 *faces,
                         int64_t F, const sm_intrinsics *K, const double *T, const void *probs, sm_dtype dt,
                         const float *scale, int c, const float *params, float *w, int32_t *rows, cudaStream_t s);
cudaError_t launch_conf_train_step(float *params, const float *feat, const float *target, int64_t n, float lr,
                                   float *grad, float *loss, cudaStream_t s, const int64_t *idx = nullptr,
                                   int64_t n_obs = 0);
void launch_conf_targets(const void *probs, sm_dtype dt, const float *scale, int c, const int32_t *rows, int64_t n,
                         const uint8_t *labels8, int64_t n_x, float *y, cudaStream_t s);
void launch_normalise(sm_rule rule, const float *acc, const uint32_t *cnt, int64_t n_x, int c, float *dist,
                      int32_t *labels, uint8_t *labels8, cudaStream_t s);
void launch_render(const int32_t *idmap, int64_t npix, const uint8_t *labels8, int64_t n_x, uint8_t *out,
                   cudaStream_t s);

// ---- kernels (mesh.cu) ----
void launch_pack_mesh(const float *verts, int64_t V, const int32_t *faces, int64_t F, float4 *verts4, int4 *faces4,
                      int32_t *err, cudaStream_t s);
// Texel layout: texinfo[f] = s | (uv origin << 16); row0 = exclusive prefix
// sum of (s^2+s)/2; *n_x_out (device int64) = total.  scratch needs
// texel_scan_scratch_bytes(F) bytes.
size_t texel_scan_scratch_bytes(int64_t F);
void launch_texel_layout(const int32_t *res, const float4 *verts4, const int4 *faces4, int64_t F, int32_t *texinfo,
                         int32_t *row0, int64_t *n_x_out, void *scratch, int32_t *err, cudaStream_t s);

}  // namespace lf

// The opaque mesh object behind the C ABI.
struct sm_mesh {
    int device = 0;
    int64_t V = 0, F = 0, n_x = 0;
    int32_t c = 0;
    sm_rule rule = SM_RULE_SUM;
    sm_weight weight = SM_WEIGHT_PIXEL;
    float alpha = 1.0f;  // image-weight mix (sm_set_weight_mix)
    int tuned_B = 0;          // frames per launch chosen by sm_autotune_batch ...
    int64_t tuned_npix = 0;   // ... for frames of this many pixels
    // work-queue fusion (sm_set_queue_shape / sm_autotune_batch): used when
    // use_queue is set, with this shape for frames of q_npix pixels (zero
    // fields take the defaults)
    int qB = 0, qL = 0, qR = 0, qS = 0;
    int64_t q_npix = 0;
    bool use_queue = false;
    bool texel_mode = false;
    bool normalised = false;

    float4 *verts = nullptr;   // V: x, y, z, 0
    float4 *bounds = nullptr;  // per 32-face cluster: min, max corner
    int4 *faces = nullptr;     // F: i0, i1, i2, valid
    int32_t *row0 = nullptr;   // F: id_t (texel mode only)
    int32_t *texinfo = nullptr;  // F: s | origin << 16 (texel mode only)
    float *acc = nullptr;      // n_x x c
    uint32_t *cnt = nullptr;   // n_x observation counts
    uint8_t *labels8 = nullptr;  // n_x labels after sm_normalise (255 = unseen)
    int32_t *err = nullptr;    // device error latch

    // scratch, grown on demand
    lf::Camera *cams = nullptr;
    int64_t cams_cap = 0;
    unsigned long long *keys = nullptr;
    int64_t keys_cap = 0;
    // a buffer in compressible memory (api.cu grow_compressible): its mapping
    // (p == nullptr: the buffer is stream-ordered device memory)
    struct VmmBlock {
        void *p = nullptr;
        size_t mapped = 0;
        unsigned long long handle = 0;
    };
    VmmBlock keys_blk, idbuf_blk, fcnt_blk;
    int32_t *clist = nullptr;   // visible-cluster lists of one raster batch
    int64_t clist_cap = 0;
    uint32_t *ccount = nullptr;  // their lengths
    int64_t ccount_cap = 0;
    int32_t *area = nullptr;     // visible-area pre-pass: per-triangle maxima
    int64_t area_cap = 0;
    int32_t *idbuf = nullptr;
    int64_t idbuf_cap = 0;
    float *wbuf = nullptr;  // one batch of per-pixel confidence weights
    int64_t wbuf_cap = 0;
    uint32_t *fcnt = nullptr;
    int64_t fcnt_cap = 0;
    uint32_t *qctr = nullptr;  // work-queue head, completion counts and abort flag
    int64_t qctr_cap = 0;

    // raster stream + events that pipeline raster(batch b+1) with scatter(batch b)
    cudaStream_t rstream = nullptr;
    cudaEvent_t ev_start = nullptr, ev_rast[2] = {nullptr, nullptr}, ev_scat[2] = {nullptr, nullptr};

    // host-streaming path (sm_fuse_render_host): copy streams (a batch's copy
    // is split over them so that several copy engines work at once), staging
    static constexpr int kCopyStreams = 4;
    cudaStream_t cstream[kCopyStreams] = {};
    cudaEvent_t ev_h2d[2][kCopyStreams] = {}, ev_free[2] = {nullptr, nullptr};
    uint8_t *hstage = nullptr;   // two batches of predictions (+ scales)
    int64_t hstage_cap = 0;      // bytes
    int32_t *hids = nullptr;     // row maps of all frames of the call
    int64_t hids_cap = 0;
    uint8_t *hlabels = nullptr;  // label images of all frames of the call
    int64_t hlabels_cap = 0;
    VmmBlock hids_blk, hlabels_blk;
    std::vector<VmmBlock> retired;  // compressible blocks replaced during a stream capture
    double *hcam = nullptr;      // N x (4 + 16) camera parameters
    int64_t hcam_cap = 0;

    // kernel timing
    bool prof = false;
    struct EvPair {
        cudaEvent_t a, b;
    };
    std::vector<EvPair> ev[SM_K_COUNT_KINDS];
    size_t ev_used[SM_K_COUNT_KINDS] = {};
    int64_t ev_kernels[SM_K_COUNT_KINDS] = {};  // kernel launches inside the used scopes
};
