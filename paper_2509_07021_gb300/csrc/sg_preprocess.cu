// preprocessSG (forward) and its adjoint.
//
// Forward, one thread per (view, Gaussian): EWA projection of the 3D Gaussian
// (Sec. 3.1) with a 0.3 px low-pass dilation, conic, 3-sigma radius, tile
// rectangle, depth key, and the view-dependent SG colour of Eq. 2 with the
// soft-pruning masks. Every quantity that decides an integer (cull, radius,
// tile rectangle, depth key) is computed with a fixed binary32 recipe:
// one IEEE round-to-nearest operation per step in a written order, no fused
// multiply-add, so it is reproducible off the GPU.
//
// Backward, one thread per Gaussian of a scene, looping over the views of
// that scene: chains dL/d(centre, conic, o', rgb) of each view back to every
// scene input and writes the sums (no atomics).
#include "sg_internal.cuh"

#include <cstring>

namespace sgk {

// ---------------------------------------------------------------------------
// parameter loads (storage type -> binary32)
// ---------------------------------------------------------------------------
template <int DT>
__device__ __forceinline__ float ldp(const void *p, int64_t i);
template <>
__device__ __forceinline__ float ldp<SG_F32>(const void *p, int64_t i) {
    return __ldg(static_cast<const float *>(p) + i);
}
template <>
__device__ __forceinline__ float ldp<SG_F16>(const void *p, int64_t i) {
    return __half2float(static_cast<const __half *>(p)[i]);
}
template <>
__device__ __forceinline__ float ldp<SG_BF16>(const void *p, int64_t i) {
    return __bfloat162float(static_cast<const __nv_bfloat16 *>(p)[i]);
}

// exactly rounded binary32 steps (never contracted into FMA)
__device__ __forceinline__ float fm(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fa(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fs(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float fdv(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ float fsq(float a) { return __fsqrt_rn(a); }

__device__ __forceinline__ int clamp_tile(float f, int n) {
    // floor'ed tile coordinate -> [0, n]; NaN -> 0
    if (f >= (float)n) return n;
    if (f > 0.f) return (int)f;
    return 0;
}

struct Geo {
    // camera-space centre
    float tx, ty, tz;
    // normalised quaternion and rotation
    float qw, qx, qy, qz, invq;
    float R[3][3];
    float M[3][3];      // R * diag(s)
    float S[3][3];      // Sigma_3D
    float ux, uy;       // t_x / t_z, t_y / t_z
    float ccx, ccy;     // guard-band clamped x, y
    float j00, j02, j11, j12;
    float A[2][3];      // J * W
    float ca, cb, cc;   // Sigma_2D entries after dilation
    float det;
    float conA, conB, conC;
    float x, y;         // projected centre (pixel index coordinates)
    float rf;           // radius (float)
    int x0, y0, x1, y1; // tile rectangle, half open
    float op;           // o' = m_g * o
    bool visible;
};

// The view-independent part of the recipe: unit quaternion, rotation R,
// M = R diag(s) and Sigma_3D = M M^T (computed once per Gaussian for all views).
struct Geo3 {
    float qw, qx, qy, qz, invq;
    float R[3][3], M[3][3], S[3][3];
};

__device__ __forceinline__ void geo3_recipe(float s0, float s1, float s2, float q0, float q1, float q2,
                                            float q3, Geo3 &g) {
    const float n2 = fa(fa(fa(fm(q0, q0), fm(q1, q1)), fm(q2, q2)), fm(q3, q3));
    g.invq = fdv(1.f, fsq(n2));
    const float w = fm(q0, g.invq), x = fm(q1, g.invq), y = fm(q2, g.invq), z = fm(q3, g.invq);
    g.qw = w; g.qx = x; g.qy = y; g.qz = z;
    g.R[0][0] = fs(1.f, fm(2.f, fa(fm(y, y), fm(z, z))));
    g.R[0][1] = fm(2.f, fs(fm(x, y), fm(w, z)));
    g.R[0][2] = fm(2.f, fa(fm(x, z), fm(w, y)));
    g.R[1][0] = fm(2.f, fa(fm(x, y), fm(w, z)));
    g.R[1][1] = fs(1.f, fm(2.f, fa(fm(x, x), fm(z, z))));
    g.R[1][2] = fm(2.f, fs(fm(y, z), fm(w, x)));
    g.R[2][0] = fm(2.f, fs(fm(x, z), fm(w, y)));
    g.R[2][1] = fm(2.f, fa(fm(y, z), fm(w, x)));
    g.R[2][2] = fs(1.f, fm(2.f, fa(fm(x, x), fm(y, y))));
    const float s[3] = {s0, s1, s2};
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) g.M[i][j] = fm(g.R[i][j], s[j]);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = i; j < 3; ++j) {
            g.S[i][j] = fa(fa(fm(g.M[i][0], g.M[j][0]), fm(g.M[i][1], g.M[j][1])),
                           fm(g.M[i][2], g.M[j][2]));
            g.S[j][i] = g.S[i][j];
        }
}

// The binary32 decision recipe for one view, given the Gaussian's Geo3.
// Fills every field of g.
__device__ __forceinline__ void project_view(const ViewDesc &vw, float px, float py, float pz, const Geo3 &g3,
                                             float opac, float gmask, Geo &g) {
    const float *V = vw.V;
    g.tx = fa(fa(fa(fm(V[0], px), fm(V[1], py)), fm(V[2], pz)), V[3]);
    g.ty = fa(fa(fa(fm(V[4], px), fm(V[5], py)), fm(V[6], pz)), V[7]);
    g.tz = fa(fa(fa(fm(V[8], px), fm(V[9], py)), fm(V[10], pz)), V[11]);
    const bool near_ok = g.tz > vw.near_plane;
    g.qw = g3.qw; g.qx = g3.qx; g.qy = g3.qy; g.qz = g3.qz; g.invq = g3.invq;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            g.R[i][j] = g3.R[i][j];
            g.M[i][j] = g3.M[i][j];
            g.S[i][j] = g3.S[i][j];
        }

    const float fx = vw.fx, fy = vw.fy;
    const float tanx = fdv(fm(0.5f, (float)vw.W), fx);
    const float tany = fdv(fm(0.5f, (float)vw.H), fy);
    const float limx = fm(1.3f, tanx), limy = fm(1.3f, tany);
    g.ux = fdv(g.tx, g.tz);
    g.uy = fdv(g.ty, g.tz);
    g.ccx = fm(fminf(limx, fmaxf(-limx, g.ux)), g.tz);
    g.ccy = fm(fminf(limy, fmaxf(-limy, g.uy)), g.tz);
    const float tz2 = fm(g.tz, g.tz);
    g.j00 = fdv(fx, g.tz);
    g.j11 = fdv(fy, g.tz);
    g.j02 = -fdv(fm(fx, g.ccx), tz2);
    g.j12 = -fdv(fm(fy, g.ccy), tz2);
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        g.A[0][j] = fa(fm(g.j00, V[0 + j]), fm(g.j02, V[8 + j]));
        g.A[1][j] = fa(fm(g.j11, V[4 + j]), fm(g.j12, V[8 + j]));
    }
    float B[2][3];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            B[i][j] = fa(fa(fm(g.A[i][0], g.S[0][j]), fm(g.A[i][1], g.S[1][j])),
                         fm(g.A[i][2], g.S[2][j]));
    g.ca = fa(fa(fa(fm(B[0][0], g.A[0][0]), fm(B[0][1], g.A[0][1])), fm(B[0][2], g.A[0][2])), 0.3f);
    g.cb = fa(fa(fm(B[0][0], g.A[1][0]), fm(B[0][1], g.A[1][1])), fm(B[0][2], g.A[1][2]));
    g.cc = fa(fa(fa(fm(B[1][0], g.A[1][0]), fm(B[1][1], g.A[1][1])), fm(B[1][2], g.A[1][2])), 0.3f);
    g.det = fs(fm(g.ca, g.cc), fm(g.cb, g.cb));
    const bool det_ok = g.det > 0.f;
    g.conA = fdv(g.cc, g.det);
    g.conB = -fdv(g.cb, g.det);
    g.conC = fdv(g.ca, g.det);
    const float mid = fm(0.5f, fa(g.ca, g.cc));
    const float lam1 = fa(mid, fsq(fmaxf(0.1f, fs(fm(mid, mid), g.det))));
    g.rf = ceilf(fm(3.f, fsq(lam1)));
    g.x = fs(fa(fm(fx, g.ux), vw.cx), 0.5f);
    g.y = fs(fa(fm(fy, g.uy), vw.cy), 0.5f);
    g.x0 = clamp_tile(floorf(fdv(fs(g.x, g.rf), 16.f)), vw.tiles_x);
    g.x1 = clamp_tile(floorf(fdv(fa(fa(g.x, g.rf), 15.f), 16.f)), vw.tiles_x);
    g.y0 = clamp_tile(floorf(fdv(fs(g.y, g.rf), 16.f)), vw.tiles_y);
    g.y1 = clamp_tile(floorf(fdv(fa(fa(g.y, g.rf), 15.f), 16.f)), vw.tiles_y);
    const bool area_ok = (g.x1 > g.x0) && (g.y1 > g.y0);
    g.op = fm(gmask, opac);
    const bool op_ok = g.op >= (1.0f / 255.0f);
    const bool finite = isfinite(g.x) && isfinite(g.y) && isfinite(g.rf) && isfinite(g.conA) &&
                        isfinite(g.conB) && isfinite(g.conC);
    g.visible = near_ok && det_ok && area_ok && op_ok && finite;
}

// The whole recipe for one view.
__device__ __forceinline__ void project_recipe(const ViewDesc &vw, float px, float py, float pz,
                                               float s0, float s1, float s2, float q0, float q1,
                                               float q2, float q3, float opac, float gmask,
                                               Geo &g) {
    Geo3 g3;
    geo3_recipe(s0, s1, s2, q0, q1, q2, q3, g3);
    project_view(vw, px, py, pz, g3, opac, gmask, g);
}

template <int DG>
__device__ __forceinline__ void load_geo(const SceneDesc &sc, int64_t g, float &px, float &py,
                                         float &pz, float &s0, float &s1, float &s2, float &q0,
                                         float &q1, float &q2, float &q3, float &o) {
    const int64_t n = sc.n;
    px = ldp<DG>(sc.means, g);
    py = ldp<DG>(sc.means, n + g);
    pz = ldp<DG>(sc.means, 2 * n + g);
    s0 = ldp<DG>(sc.scales, g);
    s1 = ldp<DG>(sc.scales, n + g);
    s2 = ldp<DG>(sc.scales, 2 * n + g);
    q0 = ldp<DG>(sc.quats, g);
    q1 = ldp<DG>(sc.quats, n + g);
    q2 = ldp<DG>(sc.quats, 2 * n + g);
    q3 = ldp<DG>(sc.quats, 3 * n + g);
    o = ldp<DG>(sc.opac, g);
}

__device__ __forceinline__ int find_block_scene(const Batch &b, uint32_t blk) {
    int lo = 0, hi = b.n_scenes - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (b.scene[mid].blk_off <= blk) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// ---------------------------------------------------------------------------
// setup: copy the batch table into the workspace, seed the counters
// ---------------------------------------------------------------------------
// The batch table travels as a kernel parameter sized for the call: the header,
// then NV views and NS scenes (only the used ones are copied on the host).
template <int NV, int NS>
struct BatchParam {
    unsigned char head[offsetof(Batch, view)];
    ViewDesc view[NV];
    SceneDesc scene[NS];
};
static_assert(offsetof(Batch, view) % 8 == 0, "batch header");

// Writes the table into the workspace, zeroes the counters and the regions the
// caller names (e.g. tile ranges, sort scratch, the backward's accumulators),
// and seeds the entry and tile counts. Block 0 writes the table and counters;
// every block zeroes its share of the regions (16-byte stores where a region
// starts on a 16-byte boundary).
template <int NV, int NS>
__global__ void __launch_bounds__(256) k_setup(const BatchParam<NV, NS> p, Batch *dst, uint64_t *counters,
                                               ZeroRegions z) {
    chain_enter();
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t nth = (uint64_t)gridDim.x * blockDim.x;
    for (int r = 0; r < ZeroRegions::N; ++r) {
        uint32_t *ptr = z.ptr[r];
        const uint64_t words = z.words[r];
        const uint32_t ev = z.even[r];
        uint64_t i0 = 0;
        if ((reinterpret_cast<uintptr_t>(ptr) & 15u) == 0u) {
            const uint64_t n4 = words / 4;
            const uint4 v = make_uint4(ev, 0u, ev, 0u);   // words 4i, 4i + 2 are even
            for (uint64_t i = tid; i < n4; i += nth) reinterpret_cast<uint4 *>(ptr)[i] = v;
            i0 = 4 * n4;
        }
        for (uint64_t i = i0 + tid; i < words; i += nth) ptr[i] = (i & 1) ? 0u : ev;
    }
    if (blockIdx.x != 0) return;
    const Batch &hb = *reinterpret_cast<const Batch *>(p.head);   // header fields only
    const int n_views = hb.n_views, n_scenes = hb.n_scenes;
    uint32_t *d = reinterpret_cast<uint32_t *>(dst);
    const uint32_t *ph = reinterpret_cast<const uint32_t *>(p.head);
    for (int i = threadIdx.x; i < (int)(offsetof(Batch, view) / 4); i += blockDim.x) d[i] = ph[i];
    const uint32_t *pv = reinterpret_cast<const uint32_t *>(p.view);
    uint32_t *dv = reinterpret_cast<uint32_t *>(&dst->view[0]);
    for (int i = threadIdx.x; i < (int)(n_views * sizeof(ViewDesc) / 4); i += blockDim.x) dv[i] = pv[i];
    const uint32_t *ps = reinterpret_cast<const uint32_t *>(p.scene);
    uint32_t *ds = reinterpret_cast<uint32_t *>(&dst->scene[0]);
    for (int i = threadIdx.x; i < (int)(n_scenes * sizeof(SceneDesc) / 4); i += blockDim.x) ds[i] = ps[i];
    if (threadIdx.x < CNT_N) counters[threadIdx.x] = 0;
    __syncthreads();
    if (threadIdx.x == 0) {
        counters[CNT_ENTRIES] = hb.n_entries;
        counters[CNT_TILES] = hb.n_tiles;
    }
}

template <int NV, int NS>
static cudaError_t setup_t(const Batch &b, Batch *dst, uint64_t *counters, const ZeroRegions &z, cudaStream_t s) {
    BatchParam<NV, NS> p;
    std::memcpy(p.head, &b, sizeof(p.head));
    std::memcpy(p.view, b.view, (size_t)b.n_views * sizeof(ViewDesc));
    std::memcpy(p.scene, b.scene, (size_t)b.n_scenes * sizeof(SceneDesc));
    // about eight 16-byte stores per thread, up to four blocks per SM
    uint64_t words = 0;
    for (int r = 0; r < ZeroRegions::N; ++r) words += z.words[r];
    const uint64_t blocks = std::min<uint64_t>(std::max<uint64_t>(div_up(words, 256 * 32), 1), 4 * 152);
    (void)launch_chain(k_setup<NV, NS>, dim3((unsigned)blocks), dim3(256), s, p, dst, counters, z);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_setup(const Batch &b, Batch *dst, uint64_t *counters, cudaStream_t s, const ZeroRegions &z) {
    static_assert(sizeof(BatchParam<SG_MAX_VIEWS, SG_MAX_SCENES>) < 32000, "batch must fit the kernel parameters");
    if (b.n_views <= 4 && b.n_scenes <= 2) return setup_t<4, 2>(b, dst, counters, z, s);
    return setup_t<SG_MAX_VIEWS, SG_MAX_SCENES>(b, dst, counters, z, s);
}

// ---------------------------------------------------------------------------
// degree-3 real spherical harmonics (the 3DGS colour the paper replaces)
// ---------------------------------------------------------------------------
// Normalisation constants from their closed forms:
//   1/(2 sqrt(pi)), sqrt(3/(4 pi)), sqrt(15/pi)/2, sqrt(5/pi)/4, sqrt(15/pi)/4,
//   sqrt(35/(2 pi))/4, sqrt(105/pi)/2, sqrt(21/(2 pi))/4, sqrt(7/pi)/4, sqrt(105/pi)/4
constexpr float SH_C0 = 0.28209479177387814f, SH_C1 = 0.4886025119029199f;
constexpr float SH_C2A = 1.0925484305920792f, SH_C2B = 0.31539156525252005f, SH_C2C = 0.5462742152960396f;
constexpr float SH_C3A = 0.5900435899266435f, SH_C3B = 2.890611442640554f, SH_C3C = 0.4570457994644658f,
                SH_C3D = 0.3731763325901154f, SH_C3E = 1.445305721320277f;

// Y_0..Y_15 at the unit direction (x, y, z), 3DGS ordering and signs.
__device__ __forceinline__ void sh3_basis(float x, float y, float z, float Y[16]) {
    const float xx = x * x, yy = y * y, zz = z * z;
    Y[0] = SH_C0;
    Y[1] = -SH_C1 * y;
    Y[2] = SH_C1 * z;
    Y[3] = -SH_C1 * x;
    Y[4] = SH_C2A * x * y;
    Y[5] = -SH_C2A * y * z;
    Y[6] = SH_C2B * (2.f * zz - xx - yy);
    Y[7] = -SH_C2A * x * z;
    Y[8] = SH_C2C * (xx - yy);
    Y[9] = -SH_C3A * y * (3.f * xx - yy);
    Y[10] = SH_C3B * x * y * z;
    Y[11] = -SH_C3C * y * (4.f * zz - xx - yy);
    Y[12] = SH_C3D * z * (2.f * zz - 3.f * xx - 3.f * yy);
    Y[13] = -SH_C3C * x * (4.f * zz - xx - yy);
    Y[14] = SH_C3E * z * (xx - yy);
    Y[15] = -SH_C3A * x * (xx - 3.f * yy);
}

// (gx, gy, gz) += sum_k w_k grad Y_k at (x, y, z), the basis polynomials
// differentiated in x, y, z as independent variables.
__device__ __forceinline__ void sh3_grad_acc(float x, float y, float z, const float w[16], float &gx,
                                             float &gy, float &gz) {
    const float xx = x * x, yy = y * y, zz = z * z;
    gy += -SH_C1 * w[1];
    gz += SH_C1 * w[2];
    gx += -SH_C1 * w[3];
    gx += SH_C2A * y * w[4];            gy += SH_C2A * x * w[4];
    gy += -SH_C2A * z * w[5];           gz += -SH_C2A * y * w[5];
    gx += -2.f * SH_C2B * x * w[6];     gy += -2.f * SH_C2B * y * w[6];     gz += 4.f * SH_C2B * z * w[6];
    gx += -SH_C2A * z * w[7];           gz += -SH_C2A * x * w[7];
    gx += 2.f * SH_C2C * x * w[8];      gy += -2.f * SH_C2C * y * w[8];
    gx += -6.f * SH_C3A * x * y * w[9]; gy += -SH_C3A * (3.f * xx - 3.f * yy) * w[9];
    gx += SH_C3B * y * z * w[10];       gy += SH_C3B * x * z * w[10];       gz += SH_C3B * x * y * w[10];
    gx += 2.f * SH_C3C * x * y * w[11]; gy += -SH_C3C * (4.f * zz - xx - 3.f * yy) * w[11];
    gz += -8.f * SH_C3C * y * z * w[11];
    gx += -6.f * SH_C3D * x * z * w[12]; gy += -6.f * SH_C3D * y * z * w[12];
    gz += SH_C3D * (6.f * zz - 3.f * xx - 3.f * yy) * w[12];
    gx += -SH_C3C * (4.f * zz - 3.f * xx - yy) * w[13]; gy += 2.f * SH_C3C * x * y * w[13];
    gz += -8.f * SH_C3C * x * z * w[13];
    gx += 2.f * SH_C3E * x * z * w[14]; gy += -2.f * SH_C3E * y * z * w[14]; gz += SH_C3E * (xx - yy) * w[14];
    gx += -SH_C3A * (3.f * xx - 3.f * yy) * w[15]; gy += 6.f * SH_C3A * x * y * w[15];
}

// Parameters of the lobes k0 .. k0 + LOBE_CHUNK - 1 of one Gaussian, loaded
// together (two lobes per round trip measured fastest: four cost registers).
// Indices past hi - 1 repeat lobe hi - 1 (in range; those values are unused).
#ifndef SG_LOBE_CHUNK
#define SG_LOBE_CHUNK 2
#endif
constexpr int LOBE_CHUNK = SG_LOBE_CHUNK;
template <int DL, int DS>
struct LobeChunk {
    float ax[LOBE_CHUNK], ay[LOBE_CHUNK], az[LOBE_CHUNK], sh[LOBE_CHUNK], m[LOBE_CHUNK];
    float a0[LOBE_CHUNK], a1[LOBE_CHUNK], a2[LOBE_CHUNK];
    __device__ __forceinline__ void load(const SceneDesc &sc, int k0, int hi) {
        const int64_t L = sc.n_lobes;
#pragma unroll
        for (int u = 0; u < LOBE_CHUNK; ++u) {
            const int k = min(k0 + u, hi - 1);
            ax[u] = ldp<DL>(sc.axis, k); ay[u] = ldp<DL>(sc.axis, L + k); az[u] = ldp<DL>(sc.axis, 2 * L + k);
            sh[u] = ldp<DS>(sc.sharp, k);
            m[u] = __ldg(sc.lmask + k);
            a0[u] = ldp<DL>(sc.amp, k); a1[u] = ldp<DL>(sc.amp, L + k); a2[u] = ldp<DL>(sc.amp, 2 * L + k);
        }
    }
};

// ---------------------------------------------------------------------------
// K1 preprocessSG
// ---------------------------------------------------------------------------
// One (view, Gaussian) entry: projection (decision recipe), colour, record and
// tile binning. The Gaussian's parameters were loaded once by the caller.
// The view-independent part of a Gaussian's SG colour: c0 and its lobe range
// (CSR bounds clamped to [0, L] so a malformed lobe_off cannot read out of range).
struct ColourBase {
    float c0[3];
    int lo, hi;
};

template <int CM>
__device__ __forceinline__ void load_colour_base(const SceneDesc &sc, int64_t g, ColourBase &cb) {
    cb.c0[0] = cb.c0[1] = cb.c0[2] = 0.f;
    cb.lo = cb.hi = 0;
    if (CM == SG_COLOR_SH3) return;
    const int64_t n = sc.n;
    cb.c0[0] = __ldg(sc.c0 + g); cb.c0[1] = __ldg(sc.c0 + n + g); cb.c0[2] = __ldg(sc.c0 + 2 * n + g);
    cb.hi = min(__ldg(sc.lobe_off + g + 1), (int)sc.n_lobes);
    cb.lo = max(0, min(__ldg(sc.lobe_off + g), cb.hi));
}

template <int DL, int DS, int CM>
__device__ __forceinline__ void preprocess_entry(const ViewDesc &vw, const SceneDesc &sc, int64_t g, float px,
                                                 float py, float pz, const Geo3 &g3, float o, float gm,
                                                 const ColourBase &cb, uint64_t e,
                                                 Rec *__restrict__ rec, uint32_t *__restrict__ tiles_touched,
                                                 uint2 *__restrict__ rect, uint32_t *__restrict__ dkey,
                                                 uint32_t *__restrict__ dval, uint8_t *__restrict__ clamp) {
    Geo G;
    project_view(vw, px, py, pz, g3, o, gm, G);
    if (!G.visible) {
        tiles_touched[e] = 0u;
        rect[e] = make_uint2(0u, 0u);
        dkey[e] = SORT_DROP_KEY;
        dval[e] = (uint32_t)e;
        return;
    }

    // SG colour (Eq. 2): view direction from the camera centre to the Gaussian
    float dx = px - vw.campos[0], dy = py - vw.campos[1], dz = pz - vw.campos[2];
    const float inv = 1.0f / sqrtf(dx * dx + dy * dy + dz * dz);
    dx *= inv; dy *= inv; dz *= inv;
    const int64_t n = sc.n, L = sc.n_lobes;
    float cr, cg, cbl;
    if (CM == SG_COLOR_SH3) {
        float Y[16];
        sh3_basis(dx, dy, dz, Y);
        float c[3] = {0.5f, 0.5f, 0.5f};
#pragma unroll
        for (int ch = 0; ch < 3; ++ch)
#pragma unroll
            for (int k = 0; k < 16; ++k) c[ch] = fmaf(Y[k], __ldg(sc.sh + (int64_t)(ch * 16 + k) * n + g), c[ch]);
        cr = c[0]; cg = c[1]; cbl = c[2];
    } else {
        cr = cb.c0[0]; cg = cb.c0[1]; cbl = cb.c0[2];
        for (int k0 = cb.lo; k0 < cb.hi; k0 += LOBE_CHUNK) {
            LobeChunk<DL, DS> lc;
            lc.load(sc, k0, cb.hi);
#pragma unroll
            for (int u = 0; u < LOBE_CHUNK; ++u) {
                if (k0 + u >= cb.hi) break;
                const float ax = lc.ax[u], ay = lc.ay[u], az = lc.az[u];
                const float ia = 1.0f / sqrtf(ax * ax + ay * ay + az * az);
                const float dot = (ax * dx + ay * dy + az * dz) * ia;
                const float wgt = lc.m[u] * expf(lc.sh[u] * (dot - 1.0f));
                cr += wgt * lc.a0[u];
                cg += wgt * lc.a1[u];
                cbl += wgt * lc.a2[u];
            }
        }
    }
    // channels clamped by max(c, 0) (not c >= 0, NaN included): the backward reads these bits
    clamp[e] = (uint8_t)((cr >= 0.f ? 0u : 1u) | (cg >= 0.f ? 0u : 2u) | (cbl >= 0.f ? 0u : 4u));
    const float reach_t = tile_reach_threshold(G.op);
    Rec r;
    r.a = make_float4(G.x, G.y, G.conA, G.conB);
    r.b = make_float4(G.conC, reach_t, G.op, fmaxf(cr, 0.f));
    r.c = make_float4(fmaxf(cg, 0.f), fmaxf(cbl, 0.f), G.rf, G.tz);
    rec[e] = r;
    // tiles of the rectangle that the alpha >= 1/255 ellipse reaches
    TileReach R;
    tile_reach_init(G.x, G.y, G.conA, G.conB, G.conC, reach_t, R);
    uint32_t touched = 0u;
    for (int ty = G.y0; ty < G.y1; ++ty) {
        int c0, c1;
        tile_reach_row(R, ty, G.x0, G.x1, c0, c1);
        touched += (uint32_t)(c1 - c0);
    }
    tiles_touched[e] = touched;
    rect[e] = make_uint2((uint32_t)G.x0 | ((uint32_t)G.x1 << 16), (uint32_t)G.y0 | ((uint32_t)G.y1 << 16));
    dkey[e] = touched ? __float_as_uint(G.tz) : SORT_DROP_KEY;   // no pair: not depth-sorted
    dval[e] = (uint32_t)e;
}

// One thread per scene Gaussian: its parameters are read once and projected
// into every view of the call that shows its scene. ONE_VIEW: no scene has
// more than one view, so the walk stops at the first (the parameters need not
// stay live across views).
#ifndef SG_PRE_MIN_BLOCKS
#define SG_PRE_MIN_BLOCKS 1
#endif
template <int DG, int DL, int DS, int CM, bool ONE_VIEW>
__global__ void __launch_bounds__(PRE_THREADS, SG_PRE_MIN_BLOCKS)
k_preprocess(const Batch *__restrict__ bp, Rec *__restrict__ rec, uint32_t *__restrict__ tiles_touched,
             uint2 *__restrict__ rect, uint32_t *__restrict__ dkey, uint32_t *__restrict__ dval,
             uint8_t *__restrict__ clamp) {
    chain_enter();
    const Batch &b = *bp;
    const int si = find_block_scene(b, blockIdx.x);
    const SceneDesc &sc = b.scene[si];
    const int64_t g = (int64_t)(blockIdx.x - sc.blk_off) * PRE_THREADS + threadIdx.x;
    if (g >= sc.n) return;
    float px, py, pz, s0, s1, s2, q0, q1, q2, q3, o;
    load_geo<DG>(sc, g, px, py, pz, s0, s1, s2, q0, q1, q2, q3, o);
    const float gm = __ldg(sc.gmask + g);
    ColourBase cb;   // issued with the geometry loads: one memory round trip fewer
    load_colour_base<CM>(sc, g, cb);
    Geo3 g3;
    geo3_recipe(s0, s1, s2, q0, q1, q2, q3, g3);
    for (int v = 0; v < b.n_views; ++v) {
        const ViewDesc &vw = b.view[v];
        if (vw.scene != si) continue;
        preprocess_entry<DL, DS, CM>(vw, sc, g, px, py, pz, g3, o, gm, cb, vw.ent_off + (uint64_t)g, rec,
                                     tiles_touched, rect, dkey, dval, clamp);
        if (ONE_VIEW) break;
    }
}

template <int DG, int DL, int DS, int CM = SG_COLOR_SG>
static cudaError_t launch_pre_t(const Batch &hb, const Batch *db, Rec *rec, uint32_t *tt, uint2 *rect,
                                uint32_t *dkey, uint32_t *dval, uint8_t *clamp, cudaStream_t s) {
    if (hb.scene_blocks == 0) return cudaSuccess;   // one block per 256 scene Gaussians
    if (hb.max_views_per_scene <= 1)
        (void)launch_chain(k_preprocess<DG, DL, DS, CM, true>, dim3(hb.scene_blocks), dim3(PRE_THREADS), s, db, rec, tt, rect, dkey, dval,
                                                                                   clamp);
    else
        (void)launch_chain(k_preprocess<DG, DL, DS, CM, false>, dim3(hb.scene_blocks), dim3(PRE_THREADS), s, db, rec, tt, rect, dkey, dval,
                                                                                    clamp);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_preprocess(const Batch &hb, const Batch *db, Rec *rec, uint32_t *tiles_touched,
                              uint2 *rect, uint32_t *dkey, uint32_t *dval, uint8_t *clamp, cudaStream_t s) {
    // all scenes of one call share storage types (checked by the API layer)
    const SceneDesc &sc = hb.scene[0];
    const int key = sc.dtype_geom * 9 + sc.dtype_lobe * 3 + sc.dtype_sharp;
    if (sc.color_model == SG_COLOR_SH3) {
        if (key != SG_F32 * 9 + SG_F32 * 3 + SG_F32) return cudaErrorInvalidValue;
        return launch_pre_t<SG_F32, SG_F32, SG_F32, SG_COLOR_SH3>(hb, db, rec, tiles_touched, rect, dkey, dval, clamp, s);
    }
    switch (key) {
        case SG_F32 * 9 + SG_F32 * 3 + SG_F32:
            return launch_pre_t<SG_F32, SG_F32, SG_F32>(hb, db, rec, tiles_touched, rect, dkey, dval, clamp, s);
        case SG_F16 * 9 + SG_F16 * 3 + SG_F16:
            return launch_pre_t<SG_F16, SG_F16, SG_F16>(hb, db, rec, tiles_touched, rect, dkey, dval, clamp, s);
        case SG_F16 * 9 + SG_F16 * 3 + SG_BF16:
            return launch_pre_t<SG_F16, SG_F16, SG_BF16>(hb, db, rec, tiles_touched, rect, dkey, dval, clamp, s);
        default:
            return cudaErrorInvalidValue;
    }
}

// ---------------------------------------------------------------------------
// K8 preprocess backward
// ---------------------------------------------------------------------------
// dg layout: planar [9][M] per entry: the blend adjoint's sums of dG dx, dG dy,
// dG dx^2, dG dx dy, dG dy^2 (dG = dL/dalpha G), then dL/do', dL/dr, dL/dg, dL/db.
// Resident blocks per SM requested for the preprocess adjoint (it is bound by
// the latency of its parameter loads, so occupancy matters more than registers).
#ifndef SG_PRE_BWD_MIN_BLOCKS
#define SG_PRE_BWD_MIN_BLOCKS 3
#endif

template <int DG, int DL, int DS, int CM>
__global__ void __launch_bounds__(PRE_THREADS, SG_PRE_BWD_MIN_BLOCKS)
k_preprocess_bwd(const Batch *__restrict__ bp, const uint32_t *__restrict__ tiles_touched,
                 const uint8_t *__restrict__ clamp, const float *__restrict__ dg, uint64_t M) {
    chain_enter();
    const Batch &b = *bp;
    const int si = find_block_scene(b, blockIdx.x);
    const SceneDesc &sc = b.scene[si];
    const int64_t g = (int64_t)(blockIdx.x - sc.blk_off) * PRE_THREADS + threadIdx.x;
    if (g >= sc.n) return;
    const int64_t n = sc.n, L = sc.n_lobes;

    float px, py, pz, s0, s1, s2, q0, q1, q2, q3, o;
    load_geo<DG>(sc, g, px, py, pz, s0, s1, s2, q0, q1, q2, q3, o);
    const float gm = __ldg(sc.gmask + g);
    const bool sh_mode = CM == SG_COLOR_SH3;
    const int hi = sh_mode ? 0 : min(__ldg(sc.lobe_off + g + 1), (int)L);
    const int lo = sh_mode ? 0 : max(0, min(__ldg(sc.lobe_off + g), hi));

    float d_mean[3] = {0.f, 0.f, 0.f}, d_scale[3] = {0.f, 0.f, 0.f}, d_q[4] = {0.f, 0.f, 0.f, 0.f};
    float d_opac = 0.f, d_gmask = 0.f, d_c0[3] = {0.f, 0.f, 0.f};
    bool first = true;   // first visible view writes lobe gradients, later views add
    const bool multi_view = b.n_views > 1;
    Geo3 g3;
    geo3_recipe(s0, s1, s2, q0, q1, q2, q3, g3);
    float dS[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};

    // With several views, the views whose entry of this Gaussian reaches a tile
    // are found first, 32 at a time, with independent loads (one memory round
    // trip instead of one per view); the others need no gradient work.
    for (int v0 = 0; v0 < b.n_views; v0 += 32) {
        // one view: view 0 when it sees this Gaussian's scene (its tile test
        // follows the eager loads below)
        uint32_t live = b.view[0].scene == si ? 1u : 0u;
        if (multi_view) {
            live = 0u;
#pragma unroll 8
            for (int i = 0; i < 32; ++i) {
                const int v = v0 + i;
                if (v < b.n_views && b.view[v].scene == si &&
                    tiles_touched[b.view[v].ent_off + (uint64_t)g] != 0u)
                    live |= 1u << i;
            }
        }
        while (live) {
            const int v = v0 + __ffs(live) - 1;
            live &= live - 1u;
            const ViewDesc &vw = b.view[v];
            const uint64_t e = vw.ent_off + (uint64_t)g;
            // With one view, every load is issued before the visibility test (the
            // latency of the test is hidden).
            const uint32_t tte = multi_view ? 1u : tiles_touched[e];
            // moments of dP = dL/dpower = dL/dalpha o' G over the entry's pixels
            // (dx, dy = pixel - centre); gop = sum dP = o' dL/do'.
            const float mdx = dg[e], mdy = dg[M + e], mdxx = dg[2 * M + e], mdxy = dg[3 * M + e],
                        mdyy = dg[4 * M + e], gop = dg[5 * M + e];
            const float grgb[3] = {dg[6 * M + e], dg[7 * M + e], dg[8 * M + e]};
            const uint32_t cl = clamp[e];
            if (tte == 0u) continue;
            // the forward's clamp max(c, 0) per channel, read back from its bits
            const float gc[3] = {(cl & 1u) ? 0.f : grgb[0], (cl & 2u) ? 0.f : grgb[1], (cl & 4u) ? 0.f : grgb[2]};

            // ---- colour (Eq. 2) ----
            float vx = px - vw.campos[0], vy = py - vw.campos[1], vz = pz - vw.campos[2];
            const float dn = sqrtf(vx * vx + vy * vy + vz * vz);
            const float idn = 1.0f / dn;
            vx *= idn; vy *= idn; vz *= idn;
            float dvx = 0.f, dvy = 0.f, dvz = 0.f;
            if (sh_mode) {
                // c = 0.5 + sum_k Y_k(v) sh_k per channel
                float Y[16];
                sh3_basis(vx, vy, vz, Y);
                float w[16];
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    w[k] = 0.f;
#pragma unroll
                    for (int ch = 0; ch < 3; ++ch)
                        w[k] = fmaf(gc[ch], __ldg(sc.sh + (int64_t)(ch * 16 + k) * n + g), w[k]);
                }
                sh3_grad_acc(vx, vy, vz, w, dvx, dvy, dvz);
                float *gsh = sc.grads.sh;
                if (gsh) {
#pragma unroll
                    for (int ch = 0; ch < 3; ++ch)
#pragma unroll
                        for (int k = 0; k < 16; ++k) {
                            float *dst = gsh + (int64_t)(ch * 16 + k) * n + g;
                            *dst = first ? Y[k] * gc[ch] : *dst + Y[k] * gc[ch];
                        }
                }
            }
            if (!sh_mode) {
                d_c0[0] += gc[0];
                d_c0[1] += gc[1];
                d_c0[2] += gc[2];
            }
            for (int k0 = lo; k0 < hi; k0 += LOBE_CHUNK) {
                LobeChunk<DL, DS> lc;
                lc.load(sc, k0, hi);
#pragma unroll
                for (int u = 0; u < LOBE_CHUNK; ++u) {
                    const int k = k0 + u;
                    if (k >= hi) break;
                    const float ax = lc.ax[u], ay = lc.ay[u], az = lc.az[u];
                    const float na = sqrtf(ax * ax + ay * ay + az * az);
                    const float ia = 1.0f / na;
                    const float mx = ax * ia, my = ay * ia, mz = az * ia;
                    const float dot = mx * vx + my * vy + mz * vz;
                    const float sh = lc.sh[u];
                    const float ex = expf(sh * (dot - 1.0f));
                    const float m = lc.m[u];
                    const float a0 = lc.a0[u], a1 = lc.a1[u], a2 = lc.a2[u];
                    const float ga = a0 * gc[0] + a1 * gc[1] + a2 * gc[2];
                    const float de = m * ga;
                    const float dd = de * ex * sh;                 // dL/d(mu_hat . v)
                    const float gmx = dd * vx, gmy = dd * vy, gmz = dd * vz;   // dL/dmu_hat
                    const float pr = mx * gmx + my * gmy + mz * gmz;
                    dvx += dd * mx; dvy += dd * my; dvz += dd * mz;
                    float ga_out[3] = {m * ex * gc[0], m * ex * gc[1], m * ex * gc[2]};
                    float gax[3] = {(gmx - mx * pr) * ia, (gmy - my * pr) * ia, (gmz - mz * pr) * ia};
                    const float gs = de * ex * (dot - 1.0f);
                    const float gml = ex * ga;
                    const sg_grads &gr = sc.grads;
                    if (first) {
                        if (gr.amp) { gr.amp[k] = ga_out[0]; gr.amp[L + k] = ga_out[1]; gr.amp[2 * L + k] = ga_out[2]; }
                        if (gr.axis) { gr.axis[k] = gax[0]; gr.axis[L + k] = gax[1]; gr.axis[2 * L + k] = gax[2]; }
                        if (gr.sharp) gr.sharp[k] = gs;
                        if (gr.lmask) gr.lmask[k] = gml;
                    } else {
                        if (gr.amp) {
                            gr.amp[k] += ga_out[0]; gr.amp[L + k] += ga_out[1]; gr.amp[2 * L + k] += ga_out[2];
                        }
                        if (gr.axis) { gr.axis[k] += gax[0]; gr.axis[L + k] += gax[1]; gr.axis[2 * L + k] += gax[2]; }
                        if (gr.sharp) gr.sharp[k] += gs;
                        if (gr.lmask) gr.lmask[k] += gml;
                    }
                }
            }
            first = false;
            // v = (p - cam) / |p - cam|
            {
                const float pr = vx * dvx + vy * dvy + vz * dvz;
                d_mean[0] += (dvx - vx * pr) * idn;
                d_mean[1] += (dvy - vy * pr) * idn;
                d_mean[2] += (dvz - vz * pr) * idn;
            }

            // ---- geometry: recompute the projection (after the colour part, so that
            // its intermediates are not live across the lobe loop) ----
            Geo G;
            project_view(vw, px, py, pz, g3, o, gm, G);
            // o' = m_g * o; a Gaussian with o' = 0 blends no pair (gop = 0)
            {
                const float dop = G.op > 0.f ? gop / G.op : 0.f;
                d_opac += gm * dop;
                d_gmask += o * dop;
            }
            // power = -(A dx^2 + C dy^2) / 2 - B dx dy and d/dx = -d/d(dx):
            // the gradients of the centre and of the conic
            const float gx = G.conA * mdx + G.conB * mdy;
            const float gy = G.conB * mdx + G.conC * mdy;
            const float gA = -0.5f * mdxx, gB = -mdxy, gC = -0.5f * mdyy;

            // ---- projected centre: x = fx t_x / t_z + cx - 0.5 ----
            const float itz = 1.0f / G.tz;
            float dtx = vw.fx * itz * gx;
            float dty = vw.fy * itz * gy;
            float dtz = -(vw.fx * G.tx * gx + vw.fy * G.ty * gy) * itz * itz;

            // ---- conic (A, B, C) = (c, -b, a) / det ----
            const float a = G.ca, bb = G.cb, c = G.cc;
            const float id2 = 1.0f / (G.det * G.det);
            const float da = (-c * c * gA + bb * c * gB - bb * bb * gC) * id2;
            const float db = (2.f * bb * c * gA - (a * c + bb * bb) * gB + 2.f * a * bb * gC) * id2;
            const float dc = (-bb * bb * gA + a * bb * gB - a * a * gC) * id2;

            // ---- Sigma_2D = A Sigma A^T (A = J W) ----
            float SA0[3], SA1[3];
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                SA0[i] = G.S[i][0] * G.A[0][0] + G.S[i][1] * G.A[0][1] + G.S[i][2] * G.A[0][2];
                SA1[i] = G.S[i][0] * G.A[1][0] + G.S[i][1] * G.A[1][1] + G.S[i][2] * G.A[1][2];
            }
            float dA0[3], dA1[3];
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                dA0[i] = 2.f * da * SA0[i] + db * SA1[i];
                dA1[i] = db * SA0[i] + 2.f * dc * SA1[i];
            }
            // symmetric gradient w.r.t. Sigma_3D, then M (Sigma = M M^T)
            float Gs[3][3];
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int j = 0; j < 3; ++j)
                    Gs[i][j] = 2.f * da * G.A[0][i] * G.A[0][j] +
                               db * (G.A[0][i] * G.A[1][j] + G.A[1][i] * G.A[0][j]) +
                               2.f * dc * G.A[1][i] * G.A[1][j];
            // dL/dSigma_3D summed over the views; chained to scale and rotation once
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int j = 0; j < 3; ++j) dS[i][j] += Gs[i][j];
            // J entries
            const float *V = vw.V;
            const float dJ00 = dA0[0] * V[0] + dA0[1] * V[1] + dA0[2] * V[2];
            const float dJ02 = dA0[0] * V[8] + dA0[1] * V[9] + dA0[2] * V[10];
            const float dJ11 = dA1[0] * V[4] + dA1[1] * V[5] + dA1[2] * V[6];
            const float dJ12 = dA1[0] * V[8] + dA1[1] * V[9] + dA1[2] * V[10];
            const float itz2 = itz * itz;
            dtz += -(vw.fx * dJ00 + vw.fy * dJ11) * itz2;
            {
                const float limx = 1.3f * (0.5f * (float)vw.W / vw.fx);
                const float limy = 1.3f * (0.5f * (float)vw.H / vw.fy);
                const bool inx = G.ux >= -limx && G.ux <= limx;
                const bool iny = G.uy >= -limy && G.uy <= limy;
                // J02 = -fx ccx / tz^2, ccx = clamp(tx/tz) tz
                const float dccx = -vw.fx * itz2 * dJ02;
                const float dccy = -vw.fy * itz2 * dJ12;
                dtz += 2.f * vw.fx * G.ccx * itz2 * itz * dJ02 + 2.f * vw.fy * G.ccy * itz2 * itz * dJ12;
                if (inx) dtx += dccx; else dtz += dccx * fminf(limx, fmaxf(-limx, G.ux));
                if (iny) dty += dccy; else dtz += dccy * fminf(limy, fmaxf(-limy, G.uy));
            }
            // t = W p + t
            d_mean[0] += V[0] * dtx + V[4] * dty + V[8] * dtz;
            d_mean[1] += V[1] * dtx + V[5] * dty + V[9] * dtz;
            d_mean[2] += V[2] * dtx + V[6] * dty + V[10] * dtz;
        }
    }

    const sg_grads &gr = sc.grads;
    // Sigma_3D = M M^T, M = R diag(s): scale and (unit, then raw) quaternion
    if (!first) {
        float dM[3][3];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int k = 0; k < 3; ++k)
                dM[i][k] = dS[i][0] * g3.M[0][k] + dS[i][1] * g3.M[1][k] + dS[i][2] * g3.M[2][k];
        const float sv[3] = {s0, s1, s2};
        float dR[3][3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            d_scale[k] = dM[0][k] * g3.R[0][k] + dM[1][k] * g3.R[1][k] + dM[2][k] * g3.R[2][k];
#pragma unroll
            for (int i = 0; i < 3; ++i) dR[i][k] = dM[i][k] * sv[k];
        }
        const float w = g3.qw, x = g3.qx, y = g3.qy, z = g3.qz;
        const float gw = 2.f * (-z * dR[0][1] + y * dR[0][2] + z * dR[1][0] - x * dR[1][2] -
                                y * dR[2][0] + x * dR[2][1]);
        const float gxq = 2.f * (y * dR[0][1] + z * dR[0][2] + y * dR[1][0] - 2.f * x * dR[1][1] -
                                 w * dR[1][2] + z * dR[2][0] + w * dR[2][1] - 2.f * x * dR[2][2]);
        const float gyq = 2.f * (-2.f * y * dR[0][0] + x * dR[0][1] + w * dR[0][2] + x * dR[1][0] +
                                 z * dR[1][2] - w * dR[2][0] + z * dR[2][1] - 2.f * y * dR[2][2]);
        const float gzq = 2.f * (-2.f * z * dR[0][0] - w * dR[0][1] + x * dR[0][2] + w * dR[1][0] -
                                 2.f * z * dR[1][1] + y * dR[1][2] + x * dR[2][0] + y * dR[2][1]);
        const float pr = w * gw + x * gxq + y * gyq + z * gzq;
        d_q[0] = (gw - w * pr) * g3.invq;
        d_q[1] = (gxq - x * pr) * g3.invq;
        d_q[2] = (gyq - y * pr) * g3.invq;
        d_q[3] = (gzq - z * pr) * g3.invq;
    }
    if (first && sh_mode && gr.sh) {   // not visible in any view: SH gradients are zero
        for (int k = 0; k < 48; ++k) gr.sh[(int64_t)k * n + g] = 0.f;
    }
    if (first) {   // not visible in any view: lobe gradients are zero
        for (int k = lo; k < hi; ++k) {
            if (gr.amp) { gr.amp[k] = 0.f; gr.amp[L + k] = 0.f; gr.amp[2 * L + k] = 0.f; }
            if (gr.axis) { gr.axis[k] = 0.f; gr.axis[L + k] = 0.f; gr.axis[2 * L + k] = 0.f; }
            if (gr.sharp) gr.sharp[k] = 0.f;
            if (gr.lmask) gr.lmask[k] = 0.f;
        }
    }
    if (gr.means) { gr.means[g] = d_mean[0]; gr.means[n + g] = d_mean[1]; gr.means[2 * n + g] = d_mean[2]; }
    if (gr.scales) { gr.scales[g] = d_scale[0]; gr.scales[n + g] = d_scale[1]; gr.scales[2 * n + g] = d_scale[2]; }
    if (gr.quats) {
        gr.quats[g] = d_q[0]; gr.quats[n + g] = d_q[1]; gr.quats[2 * n + g] = d_q[2]; gr.quats[3 * n + g] = d_q[3];
    }
    if (gr.opac) gr.opac[g] = d_opac;
    if (gr.gmask) gr.gmask[g] = d_gmask;
    if (gr.c0) { gr.c0[g] = d_c0[0]; gr.c0[n + g] = d_c0[1]; gr.c0[2 * n + g] = d_c0[2]; }
}

template <int DG, int DL, int DS, int CM = SG_COLOR_SG>
static cudaError_t launch_bwd_t(const Batch &hb, const Batch *db, const uint32_t *tt, const uint8_t *clamp,
                                const float *dg, uint64_t M, cudaStream_t s) {
    if (hb.scene_blocks == 0) return cudaSuccess;
    (void)launch_chain(k_preprocess_bwd<DG, DL, DS, CM>, dim3(hb.scene_blocks), dim3(PRE_THREADS), s, db, tt, clamp, dg, M);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_preprocess_backward(const Batch &hb, const Batch *db, const uint32_t *tiles_touched,
                                       const uint8_t *clamp, const float *dg, uint64_t M, cudaStream_t s) {
    const SceneDesc &sc = hb.scene[0];
    const int key = sc.dtype_geom * 9 + sc.dtype_lobe * 3 + sc.dtype_sharp;
    if (sc.color_model == SG_COLOR_SH3) {
        if (key != SG_F32 * 9 + SG_F32 * 3 + SG_F32) return cudaErrorInvalidValue;
        return launch_bwd_t<SG_F32, SG_F32, SG_F32, SG_COLOR_SH3>(hb, db, tiles_touched, clamp, dg, M, s);
    }
    switch (key) {
        case SG_F32 * 9 + SG_F32 * 3 + SG_F32:
            return launch_bwd_t<SG_F32, SG_F32, SG_F32>(hb, db, tiles_touched, clamp, dg, M, s);
        case SG_F16 * 9 + SG_F16 * 3 + SG_F16:
            return launch_bwd_t<SG_F16, SG_F16, SG_F16>(hb, db, tiles_touched, clamp, dg, M, s);
        case SG_F16 * 9 + SG_F16 * 3 + SG_BF16:
            return launch_bwd_t<SG_F16, SG_F16, SG_BF16>(hb, db, tiles_touched, clamp, dg, M, s);
        default:
            return cudaErrorInvalidValue;
    }
}

}  // namespace sgk
