/*
 * Label-fusion oracle: a plain, slow CPU restatement of the method of
 * "Improving Semantic Image Segmentation via Label Fusion in Semantically
 * Textured Meshes" (arXiv 2111.11103).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  The product
 * (the CUDA library) never calls it and shares no code, header, table or
 * constant with it.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fPIC -shared -pthread (no
 * -ffast-math).  -ffp-contract=off matters: the visibility raster below
 * follows a fixed sequence of IEEE-754 binary32 operations, and a fused
 * multiply-add would change its integer decisions (which triangle owns a
 * pixel).  Everything else is computed in binary64.
 *
 * What each part follows:
 *   - texel count and texel cells ............ Sec. 3.1 (texels, Fig. 3)
 *   - texel identifier ........................ Eq. (idtexel), Sec. 3.3.1,
 *                                               read as T(i+j)+j (the printed
 *                                               form collides; see below)
 *   - uv origin ............................... Sec. 3.1 (vertex whose
 *                                               interior angle is closest to
 *                                               a right angle)
 *   - row offsets id_t, row l = id_t + id_x ... Sec. 3.3.2, Eq. (texel-in-array)
 *   - renderer with z-buffer .................. Sec. 3.3.1 (projects every
 *                                               triangle with the frame's
 *                                               intrinsics/extrinsics; keeps
 *                                               the nearest)
 *   - projected-pixel sets K_x ................ Eq. (projected-pixels)
 *   - fusion rules f_sum, f_mul, f_maxsum ..... Eqs. (sum), (mul), (maxsum)
 *     and weighted forms ...................... Eqs. (w-sum), (w-mul), (w-maxsum)
 *   - weights w^(P)=1, w^(I)=1/|K_i ∩ K_x| .... Sec. 3.2.2
 *   - interpolated weight (1-a) + a/|K_i ∩ K_x|  Fig. 5a (the paper does not
 *                                               print its form; this linear
 *                                               mix is the project's reading)
 *   - texel steps s_t = max(1, ceil(g sqrt a_t)) Sec. 3.1, with a_t read as the
 *     and the visible-area pre-pass ........... largest number of pixels of
 *                                               triangle t visible in one
 *                                               frame (the paper's "area in
 *                                               pixels" is not pinned down)
 *   - L1 normalisation, argmax ................ Sec. 3.2.1
 *   - render-back of the fused labels ......... Sec. 3.2.1 (rendering the fused
 *                                               mesh from the original poses)
 *
 * The paper leaves the raster's numerics open (pixel centres, snapping, fill
 * rule, depth precision, near plane).  The readings used here are the
 * project's raster specification: pixel (x,y) is sampled at image point
 * (x,y); vertices are projected in binary32 with a fixed operation order and
 * snapped to a 1/256-pixel integer grid; coverage uses exact int64 edge
 * functions with a top-left fill rule; depth is the interpolated 1/z in
 * binary32; the nearest surface wins and an exact depth tie goes to the lower
 * triangle index; a triangle with any vertex at depth <= 0.05 is dropped.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Fusion rule and weight identifiers (the oracle's own numbering). */
enum { ORA_RULE_SUM = 0, ORA_RULE_LOGSUM = 1, ORA_RULE_MAXSUM = 2, ORA_RULE_VOTE = 3 };
enum { ORA_WEIGHT_PIXEL = 0, ORA_WEIGHT_IMAGE = 1 };

static const float ORA_Z_NEAR = 0.05f;            /* near-plane reading */
static const float ORA_SNAP_LIMIT = 536870912.0f; /* 2^29 sub-pixel units */
static const double ORA_P_MIN = 9.313225746154785e-10; /* 2^-30: log(0) guard */

/* ------------------------------------------------------------------------ */
/* Texels (Sec. 3.1, Fig. 3, Eq. idtexel)                                   */
/* ------------------------------------------------------------------------ */

/* |X_t| = (s^2 + s) / 2 texels for s steps per uv dimension (Sec. 3.1). */
int64_t ora_texel_count(int64_t s) { return (s * s + s) / 2; }

/* Texel identifier of cell (i, j), i = floor(s*u), j = floor(s*v), i + j < s.
 * Eq. (idtexel) prints T(i) + j with T(n) = n(n+1)/2, which maps (0,1) and
 * (1,0) to the same id when s = 2.  Cells with i + j = n are instead numbered
 * along their anti-diagonal: T(i + j) + j, a bijection onto [0, T(s)). */
int64_t ora_texel_id(int64_t i, int64_t j)
{
    int64_t n = i + j;
    return n * (n + 1) / 2 + j;
}

/* Cell of uv point (u, v) on a triangle with s steps: u >= 0, v >= 0,
 * u + v < 1 (Sec. 3.1).  Products and floors are binary32 so that the cell
 * decision is taken in the renderer's precision; the clamps keep points that
 * round onto the u + v = 1 edge inside the triangle. */
void ora_texel_cell(int32_t s, float u, float v, int32_t *i_out, int32_t *j_out)
{
    float fs = (float)s;
    int32_t i = (int32_t)floorf(fs * u);
    if (i > s - 1) i = s - 1;
    if (i < 0) i = 0;
    int32_t j = (int32_t)floorf(fs * v);
    if (j > s - 1 - i) j = s - 1 - i;
    if (j < 0) j = 0;
    *i_out = i;
    *j_out = j;
}

/* uv origin of a triangle: the local vertex whose interior angle is closest to
 * 90 degrees (Sec. 3.1).  |angle - 90deg| grows with |cos(angle)|, so the
 * vertex with the smallest cos^2 = dot^2 / (|e1|^2 |e2|^2) is chosen, lowest
 * local index on ties.  binary32, fixed order (the decision is an integer). */
int32_t ora_uv_origin(const float *p0, const float *p1, const float *p2)
{
    const float *p[3] = {p0, p1, p2};
    float best = 0.0f;
    int32_t best_k = 0;
    for (int k = 0; k < 3; ++k) {
        const float *a = p[k], *b = p[(k + 1) % 3], *c = p[(k + 2) % 3];
        float e1x = b[0] - a[0], e1y = b[1] - a[1], e1z = b[2] - a[2];
        float e2x = c[0] - a[0], e2y = c[1] - a[1], e2z = c[2] - a[2];
        float dot = (e1x * e2x + e1y * e2y) + e1z * e2z;
        float n1 = (e1x * e1x + e1y * e1y) + e1z * e1z;
        float n2 = (e2x * e2x + e2y * e2y) + e2z * e2z;
        float den = n1 * n2;
        float q = (den > 0.0f) ? (dot * dot) / den : 2.0f;
        if (k == 0 || q < best) {
            best = q;
            best_k = k;
        }
    }
    return best_k;
}

/* Row offsets id_t (Sec. 3.3.2): the texels of all triangles are stacked, so
 * id_t is the exclusive prefix sum of |X_t|.  s == NULL means s = 1 for every
 * triangle (gamma = 0: no subdivision, Sec. 3.1).  Writes F+1 offsets and
 * returns n_x. */
int64_t ora_row_offsets(const int32_t *s, int64_t F, int64_t *id_t)
{
    int64_t acc = 0;
    for (int64_t f = 0; f < F; ++f) {
        id_t[f] = acc;
        acc += ora_texel_count(s ? (int64_t)s[f] : 1);
    }
    id_t[F] = acc;
    return acc;
}

/* ------------------------------------------------------------------------ */
/* Renderer (Sec. 3.3.1)                                                    */
/* ------------------------------------------------------------------------ */

/* Camera set-up in binary64.  T is the 4x4 row-major camera-to-world pose
 * (camera axes x right, y down, z forward); K = (fx, fy, cx, cy).  World to
 * camera is R = Rcw^T, t = -R C.  The 3x4 matrix A maps a world point to
 * (256*fx*X/Z... numerators, Z): rows 0/1 give image coordinates times Z in
 * 1/256-pixel units, row 2 gives the camera depth Z.  Each entry is rounded to
 * binary32 once at the end. */
void ora_projection(const double *K, const double *T, float *A)
{
    double R[3][3], C[3], t[3];
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 3; ++c) R[r][c] = T[c * 4 + r];
        C[r] = T[r * 4 + 3];
    }
    for (int r = 0; r < 3; ++r) t[r] = -((R[r][0] * C[0] + R[r][1] * C[1]) + R[r][2] * C[2]);
    double fx = K[0], fy = K[1], cx = K[2], cy = K[3];
    for (int c = 0; c < 3; ++c) {
        A[c] = (float)(256.0 * (fx * R[0][c] + cx * R[2][c]));
        A[4 + c] = (float)(256.0 * (fy * R[1][c] + cy * R[2][c]));
        A[8 + c] = (float)R[2][c];
    }
    A[3] = (float)(256.0 * (fx * t[0] + cx * t[2]));
    A[7] = (float)(256.0 * (fy * t[1] + cy * t[2]));
    A[11] = (float)t[2];
}

typedef struct {
    int64_t x[3], y[3]; /* snapped vertices, after orientation fix-up */
    float iz[3];        /* binary32 1/Z per vertex */
    int32_t local[3];   /* original local index of each vertex */
    int64_t area2;      /* > 0 */
} ora_tri;

/* Projects one world vertex.  Returns 0 when the vertex is at or behind the
 * near plane or projects outside the snapping range (the triangle is then
 * dropped). */
static int ora_project_vertex(const float *A, const float *p, int64_t *xs, int64_t *ys, float *iz)
{
    float X = (A[0] * p[0] + A[1] * p[1]) + A[2] * p[2] + A[3];
    float Y = (A[4] * p[0] + A[5] * p[1]) + A[6] * p[2] + A[7];
    float Z = (A[8] * p[0] + A[9] * p[1]) + A[10] * p[2] + A[11];
    if (!(Z > ORA_Z_NEAR)) return 0;
    float xf = X / Z;
    float yf = Y / Z;
    if (!(fabsf(xf) <= ORA_SNAP_LIMIT) || !(fabsf(yf) <= ORA_SNAP_LIMIT)) return 0;
    *xs = (int64_t)rintf(xf);
    *ys = (int64_t)rintf(yf);
    *iz = 1.0f / Z;
    return 1;
}

/* Triangle set-up.  Returns 0 when the triangle is dropped (a vertex failed,
 * or zero area).  A negative area swaps the second and third vertex so that
 * the edge functions below are positive inside. */
static int ora_setup_triangle(const float *A, const float *V, const int32_t *tri, ora_tri *t)
{
    for (int k = 0; k < 3; ++k) {
        if (!ora_project_vertex(A, V + 3 * (int64_t)tri[k], &t->x[k], &t->y[k], &t->iz[k])) return 0;
        t->local[k] = k;
    }
    int64_t area2 = (t->x[1] - t->x[0]) * (t->y[2] - t->y[0]) - (t->y[1] - t->y[0]) * (t->x[2] - t->x[0]);
    if (area2 == 0) return 0;
    if (area2 < 0) {
        int64_t tx = t->x[1], ty = t->y[1];
        float tz = t->iz[1];
        t->x[1] = t->x[2]; t->y[1] = t->y[2]; t->iz[1] = t->iz[2];
        t->x[2] = tx; t->y[2] = ty; t->iz[2] = tz;
        t->local[1] = 2;
        t->local[2] = 1;
        area2 = -area2;
    }
    t->area2 = area2;
    return 1;
}

/* Edge function of vertex k at sample (px, py): (c - b) x (p - b) for the edge
 * b -> c opposite k; equals area2 at vertex k and 0 on the edge. */
static int64_t ora_edge(const ora_tri *t, int k, int64_t px, int64_t py)
{
    int b = (k + 1) % 3, c = (k + 2) % 3;
    int64_t dx = t->x[c] - t->x[b], dy = t->y[c] - t->y[b];
    return dx * (py - t->y[b]) - dy * (px - t->x[b]);
}

/* Top-left fill rule for image coordinates with y pointing down: an edge
 * whose direction has dy < 0 is a left edge, dy == 0 with dx > 0 a top edge.
 * Samples exactly on such an edge belong to the triangle. */
static int ora_top_left(const ora_tri *t, int k)
{
    int b = (k + 1) % 3, c = (k + 2) % 3;
    int64_t dx = t->x[c] - t->x[b], dy = t->y[c] - t->y[b];
    return dy < 0 || (dy == 0 && dx > 0);
}

static int ora_inside(const ora_tri *t, int64_t px, int64_t py, int64_t E[3])
{
    for (int k = 0; k < 3; ++k) {
        E[k] = ora_edge(t, k, px, py);
        if (E[k] < 0) return 0;
        if (E[k] == 0 && !ora_top_left(t, k)) return 0;
    }
    return 1;
}

/* Interpolated 1/z at a covered sample, binary32: per-vertex weights
 * w_k = (float)E_k * iz_k, numerator (w0 + w1) + w2, divided by area2. */
static float ora_inv_depth(const ora_tri *t, const int64_t E[3], float w[3], float *num_out)
{
    for (int k = 0; k < 3; ++k) w[k] = (float)E[k] * t->iz[k];
    float num = (w[0] + w[1]) + w[2];
    *num_out = num;
    return num / (float)t->area2;
}

static int64_t ora_floor_div256(int64_t a) { return (a >= 0) ? a / 256 : -((-a + 255) / 256); }
static int64_t ora_ceil_div256(int64_t a) { return -ora_floor_div256(-a); }

static uint32_t ora_float_bits(float f)
{
    uint32_t u;
    memcpy(&u, &f, sizeof u);
    return u;
}

/* Renders one frame: for every triangle, for every pixel centre in its
 * bounding box, test coverage and keep the nearest surface (z-buffer,
 * Sec. 3.3.1).  The z-buffer holds the key ((0xFFFFFFFF - bits(1/z)) << 32) |
 * triangle, so the smaller key is the nearer surface and an exact depth tie
 * goes to the lower triangle index.  Then every covered pixel gets its row
 * l = id_t + id_x (Eq. texel-in-array), with id_x from the winning triangle's
 * perspective-correct uv coordinates.
 *
 *   V: nV x 3 world vertices; faces: F x 3; s: F texel steps or NULL (s = 1);
 *   origin: F uv-origin local indices or NULL (only read where s > 1);
 *   id_t: F row offsets; K: fx, fy, cx, cy; T: 4x4 camera-to-world.
 *   idmap_out: H x W rows, -1 where no triangle covers the pixel centre.
 *   face_out (optional): H x W winning triangle, -1 for background.
 *   invz_out (optional): H x W interpolated 1/z of the winner, 0 for background.
 * Returns the number of covered pixels, or -1 on allocation failure. */
int64_t ora_render_frame(const float *V, int64_t nV, const int32_t *faces, int64_t F, const int32_t *s,
                         const int32_t *origin, const int64_t *id_t, const double *K, const double *T,
                         int32_t H, int32_t W, int32_t *idmap_out, int32_t *face_out, float *invz_out)
{
    (void)nV;
    float A[12];
    ora_projection(K, T, A);
    int64_t npix = (int64_t)H * W;
    uint64_t *zbuf = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(npix > 0 ? npix : 1));
    if (!zbuf) return -1;
    for (int64_t i = 0; i < npix; ++i) zbuf[i] = UINT64_MAX;

    for (int64_t f = 0; f < F; ++f) {
        ora_tri t;
        if (!ora_setup_triangle(A, V, faces + 3 * f, &t)) continue;
        int64_t minx = t.x[0], maxx = t.x[0], miny = t.y[0], maxy = t.y[0];
        for (int k = 1; k < 3; ++k) {
            if (t.x[k] < minx) minx = t.x[k];
            if (t.x[k] > maxx) maxx = t.x[k];
            if (t.y[k] < miny) miny = t.y[k];
            if (t.y[k] > maxy) maxy = t.y[k];
        }
        int64_t x0 = ora_ceil_div256(minx), x1 = ora_floor_div256(maxx);
        int64_t y0 = ora_ceil_div256(miny), y1 = ora_floor_div256(maxy);
        if (x0 < 0) x0 = 0;
        if (y0 < 0) y0 = 0;
        if (x1 > W - 1) x1 = W - 1;
        if (y1 > H - 1) y1 = H - 1;
        for (int64_t py = y0; py <= y1; ++py) {
            for (int64_t px = x0; px <= x1; ++px) {
                int64_t E[3];
                if (!ora_inside(&t, 256 * px, 256 * py, E)) continue;
                float w[3], num;
                float inv_z = ora_inv_depth(&t, E, w, &num);
                uint64_t key = ((uint64_t)(0xFFFFFFFFu - ora_float_bits(inv_z)) << 32) | (uint64_t)(uint32_t)f;
                if (key < zbuf[py * W + px]) zbuf[py * W + px] = key;
            }
        }
    }

    int64_t covered = 0;
    for (int64_t py = 0; py < H; ++py) {
        for (int64_t px = 0; px < W; ++px) {
            uint64_t key = zbuf[py * W + px];
            int32_t row = -1, face = -1;
            if (key != UINT64_MAX) {
                face = (int32_t)(key & 0xFFFFFFFFu);
                int32_t sf = s ? s[face] : 1;
                int64_t idx = 0;
                if (sf > 1) {
                    ora_tri t;
                    int64_t E[3];
                    float w[3], num, beta[3];
                    ora_setup_triangle(A, V, faces + 3 * (int64_t)face, &t);
                    ora_inside(&t, 256 * px, 256 * py, E);
                    ora_inv_depth(&t, E, w, &num);
                    /* perspective-correct barycentrics of the ORIGINAL local
                     * vertices: beta_k = w_k / num */
                    for (int k = 0; k < 3; ++k) beta[t.local[k]] = w[k] / num;
                    int32_t o = origin ? origin[face] : 0;
                    float u = beta[(o + 1) % 3], v = beta[(o + 2) % 3];
                    int32_t i, j;
                    ora_texel_cell(sf, u, v, &i, &j);
                    idx = ora_texel_id(i, j);
                }
                row = (int32_t)(id_t[face] + idx);
                ++covered;
            }
            idmap_out[py * W + px] = row;
            if (face_out) face_out[py * W + px] = face;
            if (invz_out) {
                uint32_t bits = (key == UINT64_MAX) ? 0u : 0xFFFFFFFFu - (uint32_t)(key >> 32);
                float fz;
                memcpy(&fz, &bits, sizeof fz);
                invz_out[py * W + px] = fz;
            }
        }
    }
    free(zbuf);
    return covered;
}

/* ------------------------------------------------------------------------ */
/* Aggregation (Sec. 3.2)                                                   */
/* ------------------------------------------------------------------------ */

/* Per-pixel contribution phi(p) of one prediction p (length c) for a rule:
 *   sum    : p                                  Eq. (sum)
 *   logsum : log p  (the product of Eq. (mul) is accumulated as a sum of
 *            logarithms; p is clamped below at 2^-30 so log 0 never occurs)
 *   maxsum : g(p), the entries equal to max p keep their value, the rest
 *            are 0 (Eq. maxsum); equality is tested on the stored values
 *   vote   : 1 at the first arg max, 0 elsewhere (one-hot vote) */
void ora_phi(int32_t rule, const float *p, int32_t c, double *out)
{
    float m = p[0];
    int32_t am = 0;
    for (int32_t j = 1; j < c; ++j) {
        if (p[j] > m) {
            m = p[j];
            am = j;
        }
    }
    for (int32_t j = 0; j < c; ++j) {
        switch (rule) {
        case ORA_RULE_SUM: out[j] = (double)p[j]; break;
        case ORA_RULE_LOGSUM: {
            double q = (double)p[j];
            out[j] = log(q > ORA_P_MIN ? q : ORA_P_MIN);
            break;
        }
        case ORA_RULE_MAXSUM: out[j] = (p[j] == m) ? (double)p[j] : 0.0; break;
        default: out[j] = (j == am) ? 1.0 : 0.0; break;
        }
    }
}

/* Per-pixel weights of one frame (Sec. 3.2.2): w^(P) = 1; w^(I) = 1 / |K_i ∩
 * K_x|, the reciprocal of how many pixels of this frame land on the same row.
 * Background pixels get weight 0.  counts is scratch of n_x entries that must
 * be zero on entry and is zero again on exit. */
void ora_frame_weights(int32_t weight, double alpha, const int32_t *idmap, int64_t npix, int64_t n_x,
                       int64_t *counts, double *w_out)
{
    (void)n_x;
    if (weight == ORA_WEIGHT_IMAGE) {
        for (int64_t k = 0; k < npix; ++k)
            if (idmap[k] >= 0) counts[idmap[k]] += 1;
    }
    for (int64_t k = 0; k < npix; ++k) {
        if (idmap[k] < 0) w_out[k] = 0.0;
        else if (weight == ORA_WEIGHT_IMAGE) w_out[k] = (1.0 - alpha) + alpha / (double)counts[idmap[k]];
        else w_out[k] = 1.0;
    }
    if (weight == ORA_WEIGHT_IMAGE) {
        for (int64_t k = 0; k < npix; ++k)
            if (idmap[k] >= 0) counts[idmap[k]] = 0;
    }
}

/* Adds a list of observations to the accumulators: for each pixel k with row
 * rows[k] >= 0, A[row][j] += w_k * phi(p_k)_j and cnt[row] += 1.  The sum runs
 * in binary64 in list order.  weights == NULL means w_k = 1. */
void ora_accumulate(int32_t rule, int64_t npix, const int32_t *rows, const double *weights, const float *probs,
                    int32_t c, double *A, int64_t *cnt)
{
    double *phi = (double *)malloc(sizeof(double) * (size_t)c);
    if (!phi) return;
    for (int64_t k = 0; k < npix; ++k) {
        int32_t l = rows[k];
        if (l < 0) continue;
        double w = weights ? weights[k] : 1.0;
        ora_phi(rule, probs + k * (int64_t)c, c, phi);
        for (int32_t j = 0; j < c; ++j) A[(int64_t)l * c + j] += w * phi[j];
        cnt[l] += 1;
    }
    free(phi);
}

/* Normalisation and class decision (Sec. 3.2.1): every fused result is L1
 * normalised; its arg max is the texel class.  For logsum the accumulator
 * holds L = sum w log p, and norm(prod p^w) = exp(L - max L) / sum exp(L - max L).
 * Rows never observed (cnt == 0) get label -1 and an all-zero distribution.
 * dist may be NULL; labels may be NULL. */
void ora_normalise(int32_t rule, const double *A, const int64_t *cnt, int64_t n_x, int32_t c, double *dist,
                   int32_t *labels)
{
    for (int64_t l = 0; l < n_x; ++l) {
        const double *a = A + l * (int64_t)c;
        if (cnt[l] == 0) {
            if (labels) labels[l] = -1;
            if (dist)
                for (int32_t j = 0; j < c; ++j) dist[l * (int64_t)c + j] = 0.0;
            continue;
        }
        int32_t am = 0;
        for (int32_t j = 1; j < c; ++j)
            if (a[j] > a[am]) am = j;
        if (labels) labels[l] = am;
        if (!dist) continue;
        double total = 0.0;
        if (rule == ORA_RULE_LOGSUM) {
            for (int32_t j = 0; j < c; ++j) total += exp(a[j] - a[am]);
            for (int32_t j = 0; j < c; ++j) dist[l * (int64_t)c + j] = exp(a[j] - a[am]) / total;
        } else {
            for (int32_t j = 0; j < c; ++j) total += a[j];
            for (int32_t j = 0; j < c; ++j) dist[l * (int64_t)c + j] = a[j] / total;
        }
    }
}

/* Render-back (Sec. 3.2.1): every pixel shows the fused class of the row it
 * sees; 255 for background pixels and rows never observed. */
void ora_render_labels(const int32_t *idmap, int64_t npix, const int32_t *labels, uint8_t *out)
{
    for (int64_t k = 0; k < npix; ++k) {
        int32_t l = idmap[k];
        out[k] = (l < 0 || labels[l] < 0) ? (uint8_t)255 : (uint8_t)labels[l];
    }
}

/* ------------------------------------------------------------------------ */
/* Whole sequences, threaded over frames                                    */
/* ------------------------------------------------------------------------ */

typedef struct {
    const float *V;
    int64_t nV;
    const int32_t *faces;
    int64_t F;
    const int32_t *s;
    const int32_t *origin;
    const int64_t *id_t;
    int64_t n_x;
    const double *K;     /* N x 4 */
    const double *T;     /* N x 16 */
    const float *probs;  /* N x H x W x c */
    int32_t N, H, W, c, rule, weight;
    double alpha;        /* weight mix of w^(I) (1: pure w^(I)) */
    int32_t *idmaps_out; /* N x H x W or NULL */
    int32_t nthreads, tid;
    double *A;           /* this thread's n_x x c */
    int64_t *cnt;        /* this thread's n_x */
    int status;
} ora_job;

static void *ora_worker(void *arg)
{
    ora_job *j = (ora_job *)arg;
    int64_t npix = (int64_t)j->H * j->W;
    int32_t *idmap = (int32_t *)malloc(sizeof(int32_t) * (size_t)npix);
    double *w = (double *)malloc(sizeof(double) * (size_t)npix);
    int64_t *counts = (int64_t *)calloc((size_t)(j->n_x > 0 ? j->n_x : 1), sizeof(int64_t));
    if (!idmap || !w || !counts) {
        j->status = -1;
        free(idmap); free(w); free(counts);
        return NULL;
    }
    for (int32_t i = j->tid; i < j->N; i += j->nthreads) {
        int32_t *dst = j->idmaps_out ? j->idmaps_out + (int64_t)i * npix : idmap;
        if (ora_render_frame(j->V, j->nV, j->faces, j->F, j->s, j->origin, j->id_t, j->K + 4 * (int64_t)i,
                             j->T + 16 * (int64_t)i, j->H, j->W, dst, NULL, NULL) < 0) {
            j->status = -1;
            break;
        }
        ora_frame_weights(j->weight, j->alpha, dst, npix, j->n_x, counts, w);
        ora_accumulate(j->rule, npix, dst, w, j->probs + (int64_t)i * npix * j->c, j->c, j->A, j->cnt);
    }
    free(idmap); free(w); free(counts);
    return NULL;
}

/* Renders and fuses frames 0..N-1 into A (n_x x c, binary64) and cnt (n_x),
 * which are overwritten.  Frames are dealt round-robin to nthreads threads,
 * each with private accumulators; the partial sums are added in thread order
 * (aggregation is permutation invariant, Sec. 3.3.2).  idmaps_out, if not NULL,
 * receives every frame's row map.  Returns 0, or -1 on allocation failure. */
int ora_fuse_sequence(const float *V, int64_t nV, const int32_t *faces, int64_t F, const int32_t *s,
                      const int32_t *origin, const int64_t *id_t, int64_t n_x, const double *K, const double *T,
                      const float *probs, int32_t N, int32_t H, int32_t W, int32_t c, int32_t rule, int32_t weight,
                      double alpha, int32_t nthreads, double *A, int64_t *cnt, int32_t *idmaps_out)
{
    if (nthreads < 1) nthreads = 1;
    if (nthreads > N && N > 0) nthreads = N;
    ora_job *jobs = (ora_job *)calloc((size_t)nthreads, sizeof(ora_job));
    pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    if (!jobs || !th) {
        free(jobs); free(th);
        return -1;
    }
    int rc = 0;
    for (int32_t t = 0; t < nthreads; ++t) {
        ora_job *j = &jobs[t];
        j->V = V; j->nV = nV; j->faces = faces; j->F = F; j->s = s; j->origin = origin; j->id_t = id_t;
        j->n_x = n_x; j->K = K; j->T = T; j->probs = probs; j->N = N; j->H = H; j->W = W; j->c = c;
        j->rule = rule; j->weight = weight; j->alpha = alpha; j->idmaps_out = idmaps_out; j->nthreads = nthreads;
        j->tid = t;
        if (t == 0) {
            j->A = A;
            j->cnt = cnt;
        } else {
            j->A = (double *)malloc(sizeof(double) * (size_t)(n_x * c > 0 ? n_x * c : 1));
            j->cnt = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n_x > 0 ? n_x : 1));
            if (!j->A || !j->cnt) rc = -1;
        }
        if (j->A) memset(j->A, 0, sizeof(double) * (size_t)(n_x * c));
        if (j->cnt) memset(j->cnt, 0, sizeof(int64_t) * (size_t)n_x);
    }
    if (rc == 0) {
        for (int32_t t = 1; t < nthreads; ++t) pthread_create(&th[t], NULL, ora_worker, &jobs[t]);
        ora_worker(&jobs[0]);
        for (int32_t t = 1; t < nthreads; ++t) pthread_join(th[t], NULL);
        for (int32_t t = 0; t < nthreads; ++t)
            if (jobs[t].status) rc = -1;
        for (int32_t t = 1; t < nthreads && rc == 0; ++t) {
            for (int64_t q = 0; q < n_x * c; ++q) A[q] += jobs[t].A[q];
            for (int64_t l = 0; l < n_x; ++l) cnt[l] += jobs[t].cnt[l];
        }
    }
    for (int32_t t = 1; t < nthreads; ++t) {
        free(jobs[t].A);
        free(jobs[t].cnt);
    }
    free(jobs);
    free(th);
    return rc;
}

typedef struct {
    const float *V;
    int64_t nV;
    const int32_t *faces;
    int64_t F;
    const int32_t *s;
    const int32_t *origin;
    const int64_t *id_t;
    const double *K, *T;
    int32_t N, H, W, nthreads, tid;
    int32_t *idmaps_out;
    int status;
} ora_rjob;

static void *ora_render_worker(void *arg)
{
    ora_rjob *j = (ora_rjob *)arg;
    int64_t npix = (int64_t)j->H * j->W;
    for (int32_t i = j->tid; i < j->N; i += j->nthreads) {
        if (ora_render_frame(j->V, j->nV, j->faces, j->F, j->s, j->origin, j->id_t, j->K + 4 * (int64_t)i,
                             j->T + 16 * (int64_t)i, j->H, j->W, j->idmaps_out + (int64_t)i * npix, NULL, NULL) < 0)
            j->status = -1;
    }
    return NULL;
}

/* Renders frames 0..N-1 (row maps only) on nthreads threads. */
int ora_render_sequence(const float *V, int64_t nV, const int32_t *faces, int64_t F, const int32_t *s,
                        const int32_t *origin, const int64_t *id_t, const double *K, const double *T, int32_t N,
                        int32_t H, int32_t W, int32_t nthreads, int32_t *idmaps_out)
{
    if (nthreads < 1) nthreads = 1;
    if (nthreads > N && N > 0) nthreads = N;
    ora_rjob *jobs = (ora_rjob *)calloc((size_t)nthreads, sizeof(ora_rjob));
    pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    if (!jobs || !th) {
        free(jobs); free(th);
        return -1;
    }
    for (int32_t t = 0; t < nthreads; ++t) {
        ora_rjob *j = &jobs[t];
        j->V = V; j->nV = nV; j->faces = faces; j->F = F; j->s = s; j->origin = origin; j->id_t = id_t;
        j->K = K; j->T = T; j->N = N; j->H = H; j->W = W; j->nthreads = nthreads; j->tid = t;
        j->idmaps_out = idmaps_out;
    }
    for (int32_t t = 1; t < nthreads; ++t) pthread_create(&th[t], NULL, ora_render_worker, &jobs[t]);
    ora_render_worker(&jobs[0]);
    for (int32_t t = 1; t < nthreads; ++t) pthread_join(th[t], NULL);
    int rc = 0;
    for (int32_t t = 0; t < nthreads; ++t)
        if (jobs[t].status) rc = -1;
    free(jobs);
    free(th);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Texel resolution from gamma (Sec. 3.1)                                   */
/* ------------------------------------------------------------------------ */

typedef struct {
    const float *V;
    int64_t nV;
    const int32_t *faces;
    int64_t F;
    const double *K, *T;
    const int64_t *id_t; /* face mode: row f = triangle f */
    int32_t N, H, W, nthreads, tid;
    int64_t *area; /* this thread's F maxima */
    int status;
} ora_ajob;

static void *ora_area_worker(void *arg)
{
    ora_ajob *j = (ora_ajob *)arg;
    int64_t npix = (int64_t)j->H * j->W;
    int32_t *idmap = (int32_t *)malloc(sizeof(int32_t) * (size_t)npix);
    int64_t *count = (int64_t *)calloc((size_t)(j->F > 0 ? j->F : 1), sizeof(int64_t));
    if (!idmap || !count) {
        j->status = -1;
        free(idmap); free(count);
        return NULL;
    }
    for (int32_t i = j->tid; i < j->N; i += j->nthreads) {
        /* face mode (one row per triangle): the row map holds the triangle */
        if (ora_render_frame(j->V, j->nV, j->faces, j->F, NULL, NULL, j->id_t, j->K + 4 * (int64_t)i,
                             j->T + 16 * (int64_t)i, j->H, j->W, idmap, NULL, NULL) < 0) {
            j->status = -1;
            break;
        }
        for (int64_t k = 0; k < npix; ++k)
            if (idmap[k] >= 0) count[idmap[k]] += 1;
        for (int64_t f = 0; f < j->F; ++f) {
            if (count[f] > j->area[f]) j->area[f] = count[f];
            count[f] = 0;
        }
    }
    free(idmap); free(count);
    return NULL;
}

/* a_t of Sec. 3.1 (read as above): for every triangle, the largest number of
 * pixels on which it is the visible surface in any one of the N frames.
 * area_out (F) is overwritten.  Frames are dealt to nthreads threads, whose
 * maxima are combined.  Returns 0, or -1 on allocation failure. */
int ora_visible_area(const float *V, int64_t nV, const int32_t *faces, int64_t F, const double *K, const double *T,
                     int32_t N, int32_t H, int32_t W, int32_t nthreads, int64_t *area_out)
{
    if (nthreads < 1) nthreads = 1;
    if (nthreads > N && N > 0) nthreads = N;
    ora_ajob *jobs = (ora_ajob *)calloc((size_t)nthreads, sizeof(ora_ajob));
    pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    int64_t *id_t = (int64_t *)malloc(sizeof(int64_t) * (size_t)(F + 1));
    int rc = (jobs && th && id_t) ? 0 : -1;
    if (id_t) ora_row_offsets(NULL, F, id_t);
    for (int32_t t = 0; t < nthreads && rc == 0; ++t) {
        ora_ajob *j = &jobs[t];
        j->V = V; j->nV = nV; j->faces = faces; j->F = F; j->K = K; j->T = T; j->id_t = id_t;
        j->N = N; j->H = H; j->W = W;
        j->nthreads = nthreads; j->tid = t;
        j->area = t == 0 ? area_out : (int64_t *)malloc(sizeof(int64_t) * (size_t)(F > 0 ? F : 1));
        if (!j->area) rc = -1;
        else memset(j->area, 0, sizeof(int64_t) * (size_t)F);
    }
    if (rc == 0) {
        for (int32_t t = 1; t < nthreads; ++t) pthread_create(&th[t], NULL, ora_area_worker, &jobs[t]);
        ora_area_worker(&jobs[0]);
        for (int32_t t = 1; t < nthreads; ++t) pthread_join(th[t], NULL);
        for (int32_t t = 0; t < nthreads; ++t)
            if (jobs[t].status) rc = -1;
        for (int32_t t = 1; t < nthreads && rc == 0; ++t)
            for (int64_t f = 0; f < F; ++f)
                if (jobs[t].area[f] > area_out[f]) area_out[f] = jobs[t].area[f];
    }
    for (int32_t t = 1; jobs && t < nthreads; ++t) free(jobs[t].area);
    free(jobs);
    free(th);
    free(id_t);
    return rc;
}

/* s_t = max(1, ceil(gamma * sqrt(a_t))) (Sec. 3.1), evaluated in binary32
 * (sqrt and product correctly rounded), the precision of the kernel that
 * takes the same integer decision. */
void ora_texel_res_from_gamma(const int64_t *area, int64_t F, float gamma, int32_t *s_out)
{
    for (int64_t f = 0; f < F; ++f) {
        const float g = gamma * sqrtf((float)area[f]);
        const float c = ceilf(g);
        s_out[f] = c < 1.0f ? 1 : (int32_t)c;
    }
}
