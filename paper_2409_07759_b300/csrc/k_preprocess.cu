// k_preprocess.cu -- projection of the frame-t active set (Eq. 1-2, the
// affine/EWA projection the paper defers to 3DGS, and the view-dependent SH
// colour of Sec. 8.1), and its backward (Alg. 1 loss.backward through the
// projection).
//
// One thread per record (view of a frame group x active Gaussian of that
// frame). Consecutive threads take consecutive active Gaussians of one view, so
// a Gaussian's parameters are read from HBM once per frame and from L2 by the
// frame's other views.
//
// The discrete quantities (culling, tile rectangle, tile count, depth key)
// follow a written-down FP32 operation sequence ("key mode": correctly
// rounded +,-,*,/,sqrt, floor and a polynomial exp, never contracted) so that
// an independent CPU implementation reproduces them bit for bit.
#include "swgs_internal.cuh"

namespace swgs {

// Real SH basis, degrees 0..3, with the (-1)^m sign convention of 3DGS.
// Constants: C0 = 1/(2 sqrt(pi)), C1 = sqrt(3/(4 pi)), C2a = sqrt(15/pi)/2,
// C2b = sqrt(5/pi)/4, C2c = sqrt(15/pi)/4, C3a = sqrt(35/(2 pi))/4,
// C3b = sqrt(105/pi)/2, C3c = sqrt(21/(2 pi))/4, C3d = sqrt(7/pi)/4,
// C3e = sqrt(105/pi)/4.
#define SH_C0 0.28209479177387814f
#define SH_C1 0.4886025119029199f
#define SH_C2A 1.0925484305920792f
#define SH_C2B 0.31539156525252005f
#define SH_C2C 0.5462742152960396f
#define SH_C3A 0.5900435899266435f
#define SH_C3B 2.890611442640554f
#define SH_C3C 0.4570457994644658f
#define SH_C3D 0.3731763325901154f
#define SH_C3E 1.445305721320277f

__device__ __forceinline__ void sh_basis(int K, float x, float y, float z, float* Y) {
    Y[0] = SH_C0;
    if (K > 1) {
        Y[1] = -SH_C1 * y;
        Y[2] = SH_C1 * z;
        Y[3] = -SH_C1 * x;
    }
    if (K > 4) {
        const float xx = x * x, yy = y * y, zz = z * z;
        Y[4] = SH_C2A * x * y;
        Y[5] = -SH_C2A * y * z;
        Y[6] = SH_C2B * (2.f * zz - xx - yy);
        Y[7] = -SH_C2A * x * z;
        Y[8] = SH_C2C * (xx - yy);
        if (K > 9) {
            Y[9] = -SH_C3A * y * (3.f * xx - yy);
            Y[10] = SH_C3B * x * y * z;
            Y[11] = -SH_C3C * y * (4.f * zz - xx - yy);
            Y[12] = SH_C3D * z * (2.f * zz - 3.f * xx - 3.f * yy);
            Y[13] = -SH_C3C * x * (4.f * zz - xx - yy);
            Y[14] = SH_C3E * z * (xx - yy);
            Y[15] = -SH_C3A * x * (xx - 3.f * yy);
        }
    }
}

// Gradient of sum_k w_k Y_k(x, y, z) with x, y, z independent.
__device__ __forceinline__ void sh_basis_grad(int K, float x, float y, float z, const float* w,
                                              float* g) {
    float gx = 0.f, gy = 0.f, gz = 0.f;
    if (K > 1) {
        gy += -SH_C1 * w[1];
        gz += SH_C1 * w[2];
        gx += -SH_C1 * w[3];
    }
    if (K > 4) {
        const float xx = x * x, yy = y * y, zz = z * z;
        gx += SH_C2A * y * w[4];
        gy += SH_C2A * x * w[4];
        gy += -SH_C2A * z * w[5];
        gz += -SH_C2A * y * w[5];
        gx += -2.f * SH_C2B * x * w[6];
        gy += -2.f * SH_C2B * y * w[6];
        gz += 4.f * SH_C2B * z * w[6];
        gx += -SH_C2A * z * w[7];
        gz += -SH_C2A * x * w[7];
        gx += 2.f * SH_C2C * x * w[8];
        gy += -2.f * SH_C2C * y * w[8];
        if (K > 9) {
            gx += -SH_C3A * 6.f * x * y * w[9];
            gy += -SH_C3A * (3.f * xx - 3.f * yy) * w[9];
            gx += SH_C3B * y * z * w[10];
            gy += SH_C3B * x * z * w[10];
            gz += SH_C3B * x * y * w[10];
            gx += SH_C3C * 2.f * x * y * w[11];
            gy += -SH_C3C * (4.f * zz - xx - 3.f * yy) * w[11];
            gz += -SH_C3C * 8.f * y * z * w[11];
            gx += -SH_C3D * 6.f * x * z * w[12];
            gy += -SH_C3D * 6.f * y * z * w[12];
            gz += SH_C3D * (6.f * zz - 3.f * xx - 3.f * yy) * w[12];
            gx += -SH_C3C * (4.f * zz - 3.f * xx - yy) * w[13];
            gy += SH_C3C * 2.f * x * y * w[13];
            gz += -SH_C3C * 8.f * x * z * w[13];
            gx += SH_C3E * 2.f * x * z * w[14];
            gy += -SH_C3E * 2.f * y * z * w[14];
            gz += SH_C3E * (xx - yy) * w[14];
            gx += -SH_C3A * (3.f * xx - 3.f * yy) * w[15];
            gy += SH_C3A * 6.f * x * y * w[15];
        }
    }
    g[0] = gx; g[1] = gy; g[2] = gz;
}

__device__ __forceinline__ int find_group(const GroupDev* groups, int n_groups, long long t) {
    int lo = 0, hi = n_groups - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (groups[mid].act_base <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Key-mode covariance Sigma = M M^T, M = R(q/|q|) diag(exp(log_scale)) (Eq. 2).
// Sg holds the 6 unique entries (00, 01, 02, 11, 12, 22).
__device__ __forceinline__ void km_sigma(const float* ls, const float* q, float* Sg) {
    const float s0 = km_exp(ls[0]), s1 = km_exp(ls[1]), s2 = km_exp(ls[2]);
    float nn = kmul(q[0], q[0]);
    nn = kadd(nn, kmul(q[1], q[1]));
    nn = kadd(nn, kmul(q[2], q[2]));
    nn = kadd(nn, kmul(q[3], q[3]));
    const float n = ksqrt(nn);
    const float w = kdiv(q[0], n), x = kdiv(q[1], n), y = kdiv(q[2], n), z = kdiv(q[3], n);
    const float xx = kmul(x, x), yy = kmul(y, y), zz = kmul(z, z);
    const float xy = kmul(x, y), xz = kmul(x, z), yz = kmul(y, z);
    const float wx = kmul(w, x), wy = kmul(w, y), wz = kmul(w, z);
    float R[9];
    R[0] = ksub(1.0f, kmul(2.0f, kadd(yy, zz)));
    R[1] = kmul(2.0f, ksub(xy, wz));
    R[2] = kmul(2.0f, kadd(xz, wy));
    R[3] = kmul(2.0f, kadd(xy, wz));
    R[4] = ksub(1.0f, kmul(2.0f, kadd(xx, zz)));
    R[5] = kmul(2.0f, ksub(yz, wx));
    R[6] = kmul(2.0f, ksub(xz, wy));
    R[7] = kmul(2.0f, kadd(yz, wx));
    R[8] = ksub(1.0f, kmul(2.0f, kadd(xx, yy)));
    float M[9];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        M[3 * i + 0] = kmul(R[3 * i + 0], s0);
        M[3 * i + 1] = kmul(R[3 * i + 1], s1);
        M[3 * i + 2] = kmul(R[3 * i + 2], s2);
    }
    const int I[6] = {0, 0, 0, 1, 1, 2}, J[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
    for (int e = 0; e < 6; ++e) {
        const int i = I[e], j = J[e];
        float a0 = kmul(M[3 * i + 0], M[3 * j + 0]);
        float a1 = kmul(M[3 * i + 1], M[3 * j + 1]);
        float a2 = kmul(M[3 * i + 2], M[3 * j + 2]);
        Sg[e] = kadd(kadd(a0, a1), a2);
    }
}

__device__ __forceinline__ float sg_at(const float* Sg, int i, int j) {
    // symmetric lookup into (00, 01, 02, 11, 12, 22)
    const int a = i < j ? i : j, b = i < j ? j : i;
    return Sg[a == 0 ? b : (a == 1 ? 2 + b : 5)];
}

struct PreArgs {
    swgs_gaussians g;
    const ViewDev* views;
    const GroupDev* groups;
    int n_groups;
    const int32_t* ids;
    long long total_active;
    int tile_w, tile_h;
    int sx, sy;  // super tile in tiles
    float near_plane;
    Records rec;
    bool sh_vec;  // SH rows read as float4: K * 3 a multiple of 4, sh 16-byte aligned
};

__device__ __forceinline__ int find_group_by_record(const GroupDev* groups, int n_groups,
                                                    long long r) {
    int lo = 0, hi = n_groups - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (groups[mid].rec_base <= r) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// One thread per record r = rec_base(group) + j * n_active + i (view j of the
// group, active Gaussian i): consecutive threads write consecutive records and
// read consecutive active ids; a Gaussian's parameters are re-read by each view
// of its frame from L2.
// The tile shape (TW x TH pixels; super tiles of SX x SY tiles) is a template
// parameter, so the tile arithmetic of the row runs folds to constants.
template <int TW, int TH>
__global__ void __launch_bounds__(256) preprocess_kernel(PreArgs a, long long n_rec,
                                                         const unsigned long long* n_dev) {
    constexpr int SX = TW == 32 ? 2 : 4, SY = TW == 32 ? 8 : 4;
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= dev_count(n_rec, n_dev)) return;
    const int gi = find_group_by_record(a.groups, a.n_groups, r);
    const GroupDev G = a.groups[gi];
    const long long off = r - G.rec_base;
    const int j = (int)(off / G.n_active), i = (int)(off - (long long)j * G.n_active);
    const ViewDev& V = a.views[G.view_begin + j];
    const long long slot = a.ids[G.act_base + i];
    const int K = (a.g.sh_degree + 1) * (a.g.sh_degree + 1);

    const float mu[3] = {a.g.means[3 * slot], a.g.means[3 * slot + 1], a.g.means[3 * slot + 2]};
    // camera transform
    float p[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        float s0 = kmul(V.R[3 * k + 0], mu[0]);
        float s1 = kmul(V.R[3 * k + 1], mu[1]);
        float s2 = kmul(V.R[3 * k + 2], mu[2]);
        p[k] = kadd(kadd(kadd(s0, s1), s2), V.t[k]);
    }
    const float z = p[2];
    int tiles = 0, supers = 0;
    short4 rect = make_short4(0, -1, 0, -1);
    float u = 0.f, v = 0.f, A = 0.f, B = 0.f, C = 0.f;
    bool culled = !(z > a.near_plane);
    if (!culled) {
        const float ls[3] = {a.g.log_scales[3 * slot], a.g.log_scales[3 * slot + 1],
                             a.g.log_scales[3 * slot + 2]};
        const float4 q4 = reinterpret_cast<const float4*>(a.g.quats)[slot];
        const float q[4] = {q4.x, q4.y, q4.z, q4.w};
        float Sg[6];
        km_sigma(ls, q, Sg);
        const float tanx = kdiv(kmul(0.5f, (float)V.W), V.fx);
        const float tany = kdiv(kmul(0.5f, (float)V.H), V.fy);
        const float limx = kmul(kGuard, tanx), limy = kmul(kGuard, tany);
        const float xz = kdiv(p[0], z), yz = kdiv(p[1], z);
        const float xzc = xz < -limx ? -limx : (xz > limx ? limx : xz);
        const float yzc = yz < -limy ? -limy : (yz > limy ? limy : yz);
        const float tx = kmul(xzc, z), ty = kmul(yzc, z);
        const float zz = kmul(z, z);
        const float J00 = kdiv(V.fx, z), J11 = kdiv(V.fy, z);
        const float J02 = -kdiv(kmul(V.fx, tx), zz);
        const float J12 = -kdiv(kmul(V.fy, ty), zz);
        float T0[3], T1[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            T0[c] = kadd(kmul(J00, V.R[c]), kmul(J02, V.R[6 + c]));
            T1[c] = kadd(kmul(J11, V.R[3 + c]), kmul(J12, V.R[6 + c]));
        }
        float U0[3], U1[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            U0[c] = kadd(kadd(kmul(T0[0], sg_at(Sg, 0, c)), kmul(T0[1], sg_at(Sg, 1, c))),
                         kmul(T0[2], sg_at(Sg, 2, c)));
            U1[c] = kadd(kadd(kmul(T1[0], sg_at(Sg, 0, c)), kmul(T1[1], sg_at(Sg, 1, c))),
                         kmul(T1[2], sg_at(Sg, 2, c)));
        }
        const float c00 = kadd(kadd(kmul(U0[0], T0[0]), kmul(U0[1], T0[1])), kmul(U0[2], T0[2]));
        const float c01 = kadd(kadd(kmul(U0[0], T1[0]), kmul(U0[1], T1[1])), kmul(U0[2], T1[2]));
        const float c11 = kadd(kadd(kmul(U1[0], T1[0]), kmul(U1[1], T1[1])), kmul(U1[2], T1[2]));
        const float ca = kadd(c00, kDilation), cb = c01, cc = kadd(c11, kDilation);
        const float det = ksub(kmul(ca, cc), kmul(cb, cb));
        if (!(det > 0.0f)) {
            culled = true;
        } else {
            const float mid = kmul(0.5f, kadd(ca, cc));
            float disc = ksub(kmul(mid, mid), det);
            disc = disc < 0.1f ? 0.1f : disc;
            const float l1 = kadd(mid, ksqrt(disc));
            const float rad = ceilf(kmul(3.0f, ksqrt(l1)));
            u = kadd(kmul(V.fx, xz), V.cx);
            v = kadd(kmul(V.fy, yz), V.cy);
            A = kdiv(cc, det);
            B = -kdiv(cb, det);
            C = kdiv(ca, det);
            const float fxlo = floorf(kdiv(ksub(u, rad), (float)TW));
            const float fxhi = floorf(kdiv(kadd(u, rad), (float)TW));
            const float fylo = floorf(kdiv(ksub(v, rad), (float)TH));
            const float fyhi = floorf(kdiv(kadd(v, rad), (float)TH));
            const int ntx = V.ntx, nty = V.nty;
            const int x0 = fxlo < 0.0f ? 0 : (fxlo > (float)ntx ? ntx : (int)fxlo);
            const int x1 = fxhi > (float)(ntx - 1) ? ntx - 1 : (fxhi < -1.0f ? -1 : (int)fxhi);
            const int y0 = fylo < 0.0f ? 0 : (fylo > (float)nty ? nty : (int)fylo);
            const int y1 = fyhi > (float)(nty - 1) ? nty - 1 : (fyhi < -1.0f ? -1 : (int)fyhi);
            // tiles of the bounding rectangle the 3-sigma ellipse reaches: one run
            // per tile row; the runs of the first kRunRows rows are kept for the
            // key emission (one byte each for offset and length)
            if (x1 >= x0) {
                const KmEllipse el = km_ellipse(A, B, C);
                const bool narrow = x1 - x0 < 255;
                uint16_t* runs = a.rec.runs + r * kRunRows;
                // super tiles holding kept tiles: per super row, the span of super
                // columns its tile rows' runs reach (a convex ellipse's rows leave
                // no gap in practice; any overcount is padded by the emission)
                int srow = -1, smin = 0, smax = -1;
                for (int ty = y0; ty <= y1; ++ty) {
                    int f = 0, l = 0;
                    const int cnt = km_row_run_fast(el, u, v, x0, x1, ty, TW, TH,
                                                    &f, &l);
                    if (ty - y0 < kRunRows && narrow)
                        runs[ty - y0] = (uint16_t)((cnt ? (f - x0) : 0) | (cnt << 8));
                    tiles += cnt;
                    if (cnt > 0) {
                        const int sr = ty / SY, c0 = f / SX, c1 = (f + cnt - 1) / SX;
                        if (sr != srow) {
                            if (smax >= smin) supers += smax - smin + 1;
                            srow = sr;
                            smin = c0;
                            smax = c1;
                        } else {
                            smin = min(smin, c0);
                            smax = max(smax, c1);
                        }
                    }
                }
                if (smax >= smin) supers += smax - smin + 1;
            }
            rect = make_short4((short)x0, (short)x1, (short)y0, (short)y1);
        }
    }
    const float opacity = 1.0f / (1.0f + __expf(-a.g.opacity_logits[slot]));
    // view-dependent colour (Sec. 8.1)
    float dx = mu[0] - V.campos[0], dy = mu[1] - V.campos[1], dz = mu[2] - V.campos[2];
    const float inv = rsqrtf(dx * dx + dy * dy + dz * dz);
    dx *= inv; dy *= inv; dz *= inv;
    float Y[kMaxShCoeffs];
    sh_basis(K, dx, dy, dz, Y);
    const float* shp = a.g.sh + slot * (long long)(K * 3);
    float col[3] = {0.f, 0.f, 0.f};
    if (a.sh_vec) {
        // 16-byte loads (K * 3 a multiple of 4, the array 16-byte aligned);
        // element e = 3 k + ch, taken in order, so each channel sums over k in
        // the same order as the scalar loop
        const float4* sh4 = reinterpret_cast<const float4*>(shp);
#pragma unroll
        for (int q = 0; q < kMaxShCoeffs * 3 / 4; ++q) {
            if (4 * q < K * 3) {
                const float4 c4 = sh4[q];
                const float c[4] = {c4.x, c4.y, c4.z, c4.w};
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    col[(4 * q + e) % 3] = fmaf(Y[(4 * q + e) / 3], c[e], col[(4 * q + e) % 3]);
            }
        }
    } else {
#pragma unroll
        for (int k = 0; k < kMaxShCoeffs; ++k) {
            if (k < K) {
                col[0] = fmaf(Y[k], shp[3 * k + 0], col[0]);
                col[1] = fmaf(Y[k], shp[3 * k + 1], col[1]);
                col[2] = fmaf(Y[k], shp[3 * k + 2], col[2]);
            }
        }
    }
    const float col0 = col[0], col1 = col[1], col2 = col[2];
    a.rec.a[r] = make_float4(u, v, opacity, z);
    a.rec.b[r] = make_float4(A, B, C, 0.f);
    a.rec.c[r] = make_float4(fmaxf(col0 + 0.5f, 0.f), fmaxf(col1 + 0.5f, 0.f),
                             fmaxf(col2 + 0.5f, 0.f), 0.f);
    a.rec.tiles[r] = culled ? 0 : tiles;
    a.rec.supers[r] = culled ? 0 : supers;
    a.rec.rect[r] = culled ? make_short4(0, -1, 0, -1) : rect;
    a.rec.depth_key[r] = (culled || tiles == 0) ? 0xffffffffu : __float_as_uint(z);
}

cudaError_t launch_preprocess(const swgs_gaussians& g, const ViewDev* views, const GroupDev* groups,
                              int n_groups, const int32_t* ids, long long total_active,
                              long long n_rec, int tile_w, int tile_h, float near_plane,
                              Records rec, cudaStream_t s, const unsigned long long* n_dev) {
    if (n_rec <= 0) return cudaSuccess;
    const int K = (g.sh_degree + 1) * (g.sh_degree + 1);
    const bool sh_vec = (K * 3) % 4 == 0 && (reinterpret_cast<uintptr_t>(g.sh) & 15u) == 0;
    PreArgs a{g, views, groups, n_groups, ids, total_active, tile_w, tile_h, super_w(tile_w),
              super_h(tile_w), near_plane, rec, sh_vec};
    note_launch();
    const int blocks = div_up(n_rec, 256);
    if (tile_w == 16 && tile_h == 16)
        preprocess_kernel<16, 16><<<blocks, 256, 0, s>>>(a, n_rec, n_dev);
    else if (tile_w == 8 && tile_h == 8)
        preprocess_kernel<8, 8><<<blocks, 256, 0, s>>>(a, n_rec, n_dev);
    else if (tile_w == 32 && tile_h == 8)
        preprocess_kernel<32, 8><<<blocks, 256, 0, s>>>(a, n_rec, n_dev);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Backward: grad2d (du, dv, dA, dB, dC, dopacity, dr, dg, db per record) to
// the raw parameters, summed over the views of the group, frozen skipped.
// ---------------------------------------------------------------------------
struct PreBwdArgs {
    swgs_gaussians g;
    swgs_gaussians grads;
    const ViewDev* views;
    const GroupDev* groups;
    int n_groups;
    const int32_t* ids;
    long long total_active;
    const float* grad2d;
    bool reg;      // regulariser weights in the groups
    float* loss;   // regulariser value added here (or null)
    const unsigned long long* n_dev;  // deferred sizing: the true total_active
    bool sh_vec;  // SH rows of values and gradients as float4 (both 16-byte aligned)
};

// Alg. 1 reg(): with w_o = opacity_reg vc / (V n), w_s = scale_reg vc / (3 V n)
// for a frame of n active Gaussians seen by vc of the V views, a Gaussian adds
// w_o sigmoid(logit) + w_s sum_c exp(log_scale_c) to the loss (frozen ones
// too: they count in the means) and, unless frozen, w_o sigmoid (1 - sigmoid)
// to its logit gradient and w_s exp(log_scale_c) to its log-scale gradients.
// Summed over the block first: one atomic per block, not per warp, on the
// single loss word (same-address atomics serialise in L2). Every thread of the
// block must call it.
__device__ __forceinline__ void reg_loss_add(float v, float* loss) {
    __shared__ float part[4];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        float s = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += part[w];
        if (s != 0.f) atomicAdd(loss, s);
    }
}

// At least 4 blocks of 128 per SM (128 registers, a small spill): 201 registers
// unbounded (2 blocks), 168 with the SH coefficients read where used (3 blocks);
// 5 and 6 blocks spill more than they gain (measured).
__global__ void __launch_bounds__(128, 4) preprocess_bwd_kernel(PreBwdArgs a) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool in = t < dev_count(a.total_active, a.n_dev);
    const int gi = in ? find_group(a.groups, a.n_groups, t) : 0;
    const long long slot = in ? a.ids[t] : 0;
    if (a.reg && a.loss) {
        float v = 0.f;
        if (in) {
            const GroupDev& G0 = a.groups[gi];
            const float op = 1.0f / (1.0f + __expf(-a.g.opacity_logits[slot]));
            v = G0.reg_o * op;
#pragma unroll
            for (int k = 0; k < 3; ++k) v += G0.reg_s * __expf(a.g.log_scales[3 * slot + k]);
        }
        reg_loss_add(v, a.loss);
    }
    if (!in) return;
    const GroupDev G = a.groups[gi];
    const int i = (int)(t - G.act_base);
    if (a.g.frozen && a.g.frozen[slot]) return;
    const int K = (a.g.sh_degree + 1) * (a.g.sh_degree + 1);

    const float mu[3] = {a.g.means[3 * slot], a.g.means[3 * slot + 1], a.g.means[3 * slot + 2]};
    float s[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) s[k] = __expf(a.g.log_scales[3 * slot + k]);
    const float4 q4 = reinterpret_cast<const float4*>(a.g.quats)[slot];
    const float qn2 = q4.x * q4.x + q4.y * q4.y + q4.z * q4.z + q4.w * q4.w;
    const float qinv = rsqrtf(qn2);
    const float w = q4.x * qinv, x = q4.y * qinv, y = q4.z * qinv, zq = q4.w * qinv;
    float Rq[3][3] = {
        {1.f - 2.f * (y * y + zq * zq), 2.f * (x * y - w * zq), 2.f * (x * zq + w * y)},
        {2.f * (x * y + w * zq), 1.f - 2.f * (x * x + zq * zq), 2.f * (y * zq - w * x)},
        {2.f * (x * zq - w * y), 2.f * (y * zq + w * x), 1.f - 2.f * (x * x + y * y)}};
    float M[3][3], Sg[3][3];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) M[r][c] = Rq[r][c] * s[c];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) Sg[r][c] = M[r][0] * M[c][0] + M[r][1] * M[c][1] + M[r][2] * M[c][2];
    const float opacity = 1.0f / (1.0f + __expf(-a.g.opacity_logits[slot]));
    // the SH coefficients are read where used, once for a view's colour and once
    // for its gradients (L1 hits after the first view), not held in registers:
    // the gradient sums already take 3K of them
    const float* shp = a.g.sh + slot * (long long)(K * 3);
    const bool sh_vec = a.sh_vec;
    auto sh4 = [&](int q) {  // coefficients 4q .. 4q + 3 (zero past 3K)
        if (sh_vec) return reinterpret_cast<const float4*>(shp)[q];
        float c[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) c[t] = 4 * q + t < K * 3 ? shp[4 * q + t] : 0.f;
        return make_float4(c[0], c[1], c[2], c[3]);
    };

    float gmu[3] = {0.f, 0.f, 0.f};
    float GS[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
    float glogit = 0.f;
    float gsh[kMaxShCoeffs * 3];
#pragma unroll
    for (int k = 0; k < kMaxShCoeffs * 3; ++k) gsh[k] = 0.f;
    bool any = false;

    for (int j = 0; j < G.view_count; ++j) {
        const ViewDev& V = a.views[G.view_begin + j];
        const long long r = (long long)G.rec_base + (long long)j * G.n_active + i;
        const float4 g0 = reinterpret_cast<const float4*>(a.grad2d)[3 * r + 0];
        const float4 g1 = reinterpret_cast<const float4*>(a.grad2d)[3 * r + 1];
        const float4 g2 = reinterpret_cast<const float4*>(a.grad2d)[3 * r + 2];
        const float gu = g0.x, gv = g0.y, gA = g0.z, gB = g0.w, gC = g1.x, go = g1.y;
        const float gcol[3] = {g1.z, g1.w, g2.x};
        if (gu == 0.f && gv == 0.f && gA == 0.f && gB == 0.f && gC == 0.f && go == 0.f &&
            gcol[0] == 0.f && gcol[1] == 0.f && gcol[2] == 0.f)
            continue;
        any = true;
        glogit += go * opacity * (1.f - opacity);
        // colour
        {
            float dx = mu[0] - V.campos[0], dy = mu[1] - V.campos[1], dz = mu[2] - V.campos[2];
            const float dist = sqrtf(dx * dx + dy * dy + dz * dz);
            const float inv = 1.f / dist;
            dx *= inv; dy *= inv; dz *= inv;
            float Y[kMaxShCoeffs];
            sh_basis(K, dx, dy, dz, Y);
            // the view's colour, summed over k in the forward's order per channel
            float acc[3] = {0.f, 0.f, 0.f};
#pragma unroll
            for (int q = 0; q < kMaxShCoeffs * 3 / 4; ++q) {
                if (4 * q >= K * 3) break;
                const float4 c4 = sh4(q);
                const float c[4] = {c4.x, c4.y, c4.z, c4.w};
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const int e = 4 * q + t;
                    if (e < K * 3) acc[e % 3] = fmaf(Y[e / 3], c[t], acc[e % 3]);
                }
            }
            float gc[3];
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) gc[ch] = (acc[ch] + 0.5f > 0.f) ? gcol[ch] : 0.f;
            float wgt[kMaxShCoeffs];
#pragma unroll
            for (int k = 0; k < kMaxShCoeffs; ++k) wgt[k] = 0.f;
#pragma unroll
            for (int q = 0; q < kMaxShCoeffs * 3 / 4; ++q) {
                if (4 * q >= K * 3) break;
                const float4 c4 = sh4(q);
                const float c[4] = {c4.x, c4.y, c4.z, c4.w};
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const int e = 4 * q + t;
                    if (e < K * 3) {
                        gsh[e] += Y[e / 3] * gc[e % 3];
                        wgt[e / 3] += gc[e % 3] * c[t];
                    }
                }
            }
            float gd[3];
            sh_basis_grad(K, dx, dy, dz, wgt, gd);
            const float dd = dx * gd[0] + dy * gd[1] + dz * gd[2];
            gmu[0] += (gd[0] - dx * dd) * inv;
            gmu[1] += (gd[1] - dy * dd) * inv;
            gmu[2] += (gd[2] - dz * dd) * inv;
        }
        // geometry
        float p[3];
#pragma unroll
        for (int k = 0; k < 3; ++k)
            p[k] = V.R[3 * k] * mu[0] + V.R[3 * k + 1] * mu[1] + V.R[3 * k + 2] * mu[2] + V.t[k];
        const float z = p[2], iz = 1.f / z, iz2 = iz * iz;
        const float limx = kGuard * (0.5f * V.W / V.fx), limy = kGuard * (0.5f * V.H / V.fy);
        const float xz = p[0] * iz, yz = p[1] * iz;
        const float clx = xz < -limx ? -1.f : (xz > limx ? 1.f : 0.f);
        const float cly = yz < -limy ? -1.f : (yz > limy ? 1.f : 0.f);
        const float tx = (clx != 0.f ? clx * limx : xz) * z;
        const float ty = (cly != 0.f ? cly * limy : yz) * z;
        const float J00 = V.fx * iz, J11 = V.fy * iz;
        const float J02 = -V.fx * tx * iz2, J12 = -V.fy * ty * iz2;
        float T0[3], T1[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            T0[c] = J00 * V.R[c] + J02 * V.R[6 + c];
            T1[c] = J11 * V.R[3 + c] + J12 * V.R[6 + c];
        }
        float TS0[3], TS1[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            TS0[c] = T0[0] * Sg[0][c] + T0[1] * Sg[1][c] + T0[2] * Sg[2][c];
            TS1[c] = T1[0] * Sg[0][c] + T1[1] * Sg[1][c] + T1[2] * Sg[2][c];
        }
        const float ca = TS0[0] * T0[0] + TS0[1] * T0[1] + TS0[2] * T0[2] + kDilation;
        const float cb = TS0[0] * T1[0] + TS0[1] * T1[1] + TS0[2] * T1[2];
        const float cc = TS1[0] * T1[0] + TS1[1] * T1[1] + TS1[2] * T1[2] + kDilation;
        const float idet = 1.f / (ca * cc - cb * cb);
        const float Ai = cc * idet, Bi = -cb * idet, Ci = ca * idet;
        // d(conic) -> d(cov): -Ci Gc Ci, Gc = [[gA, gB/2], [gB/2, gC]]
        const float X00 = Ai * gA + Bi * 0.5f * gB, X01 = Ai * 0.5f * gB + Bi * gC;
        const float X10 = Bi * gA + Ci * 0.5f * gB, X11 = Bi * 0.5f * gB + Ci * gC;
        const float g00 = -(X00 * Ai + X01 * Bi);
        const float g01 = -(X00 * Bi + X01 * Ci);
        const float g11 = -(X10 * Bi + X11 * Ci);
        // cov = T Sigma T^T
#pragma unroll
        for (int r2 = 0; r2 < 3; ++r2)
#pragma unroll
            for (int c = 0; c < 3; ++c)
                GS[r2][c] += g00 * T0[r2] * T0[c] + g01 * (T0[r2] * T1[c] + T1[r2] * T0[c]) +
                             g11 * T1[r2] * T1[c];
        float GT0[3], GT1[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            GT0[c] = 2.f * (g00 * TS0[c] + g01 * TS1[c]);
            GT1[c] = 2.f * (g01 * TS0[c] + g11 * TS1[c]);
        }
        const float GJ00 = GT0[0] * V.R[0] + GT0[1] * V.R[1] + GT0[2] * V.R[2];
        const float GJ02 = GT0[0] * V.R[6] + GT0[1] * V.R[7] + GT0[2] * V.R[8];
        const float GJ11 = GT1[0] * V.R[3] + GT1[1] * V.R[4] + GT1[2] * V.R[5];
        const float GJ12 = GT1[0] * V.R[6] + GT1[1] * V.R[7] + GT1[2] * V.R[8];
        float gp0 = 0.f, gp1 = 0.f, gz = 0.f;
        gz += -GJ00 * V.fx * iz2 - GJ11 * V.fy * iz2 + GJ02 * 2.f * V.fx * tx * iz2 * iz +
              GJ12 * 2.f * V.fy * ty * iz2 * iz;
        const float gtx = -GJ02 * V.fx * iz2, gty = -GJ12 * V.fy * iz2;
        if (clx == 0.f) gp0 += gtx; else gz += gtx * clx * limx;
        if (cly == 0.f) gp1 += gty; else gz += gty * cly * limy;
        gp0 += gu * V.fx * iz;
        gz += -gu * V.fx * p[0] * iz2;
        gp1 += gv * V.fy * iz;
        gz += -gv * V.fy * p[1] * iz2;
#pragma unroll
        for (int c = 0; c < 3; ++c) gmu[c] += V.R[c] * gp0 + V.R[3 + c] * gp1 + V.R[6 + c] * gz;
    }
    if (!any) {
        if (a.reg) {
            red_add(&a.grads.opacity_logits[slot], G.reg_o * opacity * (1.f - opacity));
#pragma unroll
            for (int k = 0; k < 3; ++k) red_add(&a.grads.log_scales[3 * slot + k], G.reg_s * s[k]);
        }
        return;
    }
    if (a.reg) {
        glogit += G.reg_o * opacity * (1.f - opacity);
    }
    // Sigma = M M^T, M = Rq diag(s)
    float GM[3][3];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c)
            GM[r][c] = (GS[r][0] + GS[0][r]) * M[0][c] + (GS[r][1] + GS[1][r]) * M[1][c] +
                       (GS[r][2] + GS[2][r]) * M[2][c];
    float GR[3][3], gls[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        float gsc = 0.f;
#pragma unroll
        for (int r = 0; r < 3; ++r) { gsc += Rq[r][c] * GM[r][c]; GR[r][c] = s[c] * GM[r][c]; }
        gls[c] = gsc * s[c] + (a.reg ? G.reg_s * s[c] : 0.f);
    }
    float gq[4];
    gq[0] = 2.f * (-zq * GR[0][1] + y * GR[0][2] + zq * GR[1][0] - x * GR[1][2] - y * GR[2][0] +
                   x * GR[2][1]);
    gq[1] = 2.f * (y * GR[0][1] + zq * GR[0][2] + y * GR[1][0] - 2.f * x * GR[1][1] - w * GR[1][2] +
                   zq * GR[2][0] + w * GR[2][1] - 2.f * x * GR[2][2]);
    gq[2] = 2.f * (-2.f * y * GR[0][0] + x * GR[0][1] + w * GR[0][2] + x * GR[1][0] +
                   zq * GR[1][2] - w * GR[2][0] + zq * GR[2][1] - 2.f * y * GR[2][2]);
    gq[3] = 2.f * (-2.f * zq * GR[0][0] - w * GR[0][1] + x * GR[0][2] + w * GR[1][0] -
                   2.f * zq * GR[1][1] + y * GR[1][2] + x * GR[2][0] + y * GR[2][1]);
    const float qn[4] = {w, x, y, zq};
    const float dq = w * gq[0] + x * gq[1] + y * gq[2] + zq * gq[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) red_add(&a.grads.means[3 * slot + k], gmu[k]);
#pragma unroll
    for (int k = 0; k < 3; ++k) red_add(&a.grads.log_scales[3 * slot + k], gls[k]);
#pragma unroll
    for (int k = 0; k < 4; ++k) red_add(&a.grads.quats[4 * slot + k], (gq[k] - qn[k] * dq) * qinv);
    red_add(&a.grads.opacity_logits[slot], glogit);
    float* gshp = a.grads.sh + slot * (long long)(K * 3);
    if (a.sh_vec) {  // one 16-byte reduction per four coefficients
#pragma unroll
        for (int q = 0; q < kMaxShCoeffs * 3 / 4; ++q)
            if (4 * q < K * 3)
                red_add_v4(&gshp[4 * q], gsh[4 * q], gsh[4 * q + 1], gsh[4 * q + 2],
                           gsh[4 * q + 3]);
    } else {
#pragma unroll
        for (int k = 0; k < kMaxShCoeffs * 3; ++k)
            if (k < K * 3) red_add(&gshp[k], gsh[k]);
    }
}

cudaError_t launch_preprocess_bwd(const swgs_gaussians& g, const swgs_gaussians& grads,
                                  const ViewDev* views, const GroupDev* groups, int n_groups,
                                  const int32_t* ids, long long total_active,
                                  const float* grad2d, bool reg, float* loss, cudaStream_t s,
                                  const unsigned long long* n_dev) {
    if (total_active <= 0) return cudaSuccess;
    const int K = (g.sh_degree + 1) * (g.sh_degree + 1);
    const bool sh_vec = (K * 3) % 4 == 0 && (reinterpret_cast<uintptr_t>(g.sh) & 15u) == 0 &&
                        (reinterpret_cast<uintptr_t>(grads.sh) & 15u) == 0;
    PreBwdArgs a{g, grads, views, groups, n_groups, ids, total_active, grad2d, reg, loss, n_dev,
                 sh_vec};
    note_launch();
    preprocess_bwd_kernel<<<div_up(total_active, 128), 128, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace swgs
