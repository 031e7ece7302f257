// Adjoint of the FFT method: the gradient of a loss L(I) with respect to the displacements
// (Taylor path, Section III C) or the moments (Section III D), given dL/dI on the grid.
// The paper has no adjoint; this is the chain rule of its forward equations, TOTAL mode.
//
// Displacive.  F_m(G) = sum_mu phi_mu(G) sum_t c_t(G) M'_{m,mu,t}(k) with the stored transforms
// M' = i^n FFT(field_t), field_t = w (v1^a/a!)(v2^b/b!)(v3^c/c!), v_j = gs_j b*_j . u (the
// displacement on the reciprocal axes, scaled), c_t = x1^a x2^b x3^c with x_j = g_j / gs_j, and
// I = sum_m |F_m|^2 / (M N).  Hence
//     dL/dfield_{m,mu,t}(R) = Re[ i^n sum_k exp(ik.R) Z_{m,mu,t}(k) ],
//     Z_{m,mu,t}(k) = (2/(M N)) sum_{H: H+k in grid} dL/dI(G) conj(F_m(G)) phi_mu(G) c_t(G),
//     dL/dv_j(R) = w sum_t dL/dfield_t(R) field_{t - e_j}(R) / w,
//     dL/du_alpha(R) = sum_j gs_j b*_{j,alpha} dL/dv_j(R),
// because d(v^a/a!)/dv = v^(a-1)/(a-1)!.  Magnetic: I = C sum_m F^H P F / (M N) with
// P = 1 - G^ G^T (2/3 at G = 0), so dL/dM_{m,mu,alpha}(R) = Re[sum_k exp(ik.R) Z_{m,mu,alpha}(k)],
// Z = (2C/(M N)) sum_H dL/dI conj((P F)_alpha) phi_mu.
//
// Steps: the forward pass writing F (api.cu), the transposed recombination below (one CTA
// per k of the full k space; threads own monomials, zones are swept in chunks staged in shared
// memory), a complex FFT with the same +i sign keeping the real part, and a per-atom gather.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "api_internal.h"
#include "fft_reg.cuh"
#include "internal.h"

using namespace ds;

namespace ds {
// adjoint_sf.cu: Z of the displacive adjoint by the transposed sum factorisation (FP32); false when
// it does not apply (order above 31, zone boxes wider than 17)
bool adjoint_z_disp_sf(const RecombParams<float> &p, const float *dLdI, const float2 *F, int P, double scale,
                       float2 *Z, cudaStream_t s);
}  // namespace ds

namespace {

__device__ __forceinline__ int fdiv(int a, int b) {
    int q = a / b;
    if ((a % b != 0) && ((a < 0) != (b < 0))) --q;
    return q;
}

// complex fields [f][k1][k2][k3] (full) -> planes transformed along axes 3 and 2
template <typename T>
__global__ void k_fft_planes_c(Geometry g, const c_t<T> *in, int f0, c_t<T> *work, const c_t<T> *W2g, const c_t<T> *W3g) {
    using C = c_t<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n1 = g.n[0], n2 = g.n[1], n3 = g.n[2];
    C *W2 = (C *)smem_raw;
    C *W3 = W2 + n2;
    C *bufA = W3 + n3;
    C *bufB = bufA + (size_t)n2 * n3;
    for (int i = threadIdx.x; i < n2; i += blockDim.x) W2[i] = W2g[i];
    for (int i = threadIdx.x; i < n3; i += blockDim.x) W3[i] = W3g[i];
    const int fl = blockIdx.x / n1, k1 = blockIdx.x - fl * n1;
    const C *src = in + ((size_t)(f0 + fl) * n1 + k1) * n2 * n3;
    for (int i = threadIdx.x; i < n2 * n3; i += blockDim.x) bufA[i] = src[i];
    __syncthreads();
    C *r = fft_lines<T>(bufA, bufB, g.ax[2], W3, n2, n2, n3, 0, 1);
    C *o = (r == bufA) ? bufB : bufA;
    C *r2 = fft_lines<T>(r, o, g.ax[1], W2, n3, n3, 1, 0, n3);
    C *dst = work + ((size_t)fl * n1 + k1) * n2 * n3;
    for (int i = threadIdx.x; i < n2 * n3; i += blockDim.x) dst[i] = r2[i];
}

// columns along axis 1, output Re(i^rot x) as real fields [f][R1][R2][R3]
template <typename T>
__global__ void k_fft_columns_re(Geometry g, int f0, int cb, const c_t<T> *work, T *out, const c_t<T> *W1g,
                                 const int4 *terms, int nT) {
    using C = c_t<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n1 = g.n[0];
    const int ncol = g.n[1] * g.n[2];
    C *W1 = (C *)smem_raw;
    C *bufA = W1 + n1;
    C *bufB = bufA + (size_t)n1 * cb;
    for (int i = threadIdx.x; i < n1; i += blockDim.x) W1[i] = W1g[i];
    const int nchunk = (ncol + cb - 1) / cb;
    const int fl = blockIdx.x / nchunk;
    const int c0 = (blockIdx.x - fl * nchunk) * cb;
    const C *in = work + (size_t)fl * n1 * ncol;
    for (int idx = threadIdx.x; idx < n1 * cb; idx += blockDim.x) {
        const int r1 = idx / cb, c = idx - r1 * cb;
        bufA[idx] = (c0 + c < ncol) ? in[(size_t)r1 * ncol + c0 + c] : mk<T>(T(0), T(0));
    }
    __syncthreads();
    C *res = fft_lines<T>(bufA, bufB, g.ax[0], W1, cb, cb, 1, 0, cb);
    const int f = f0 + fl;
    const int rot = terms ? terms[f % nT].w : 0;
    T *o = out + (size_t)f * g.ncell;
    for (int idx = threadIdx.x; idx < n1 * cb; idx += blockDim.x) {
        const int r1 = idx / cb, c = idx - r1 * cb;
        if (c0 + c < ncol) o[(size_t)r1 * ncol + c0 + c] = cipow(res[idx], rot).x;
    }
}

// FP32 fields of 32^3 cells: lines of 32 points in one thread's registers (compile-time twiddles).
// Planes: a CTA stages four 32 x 32 planes (rows padded to 33: conflict-free rows and columns), a
// warp transforms one plane, a thread a row (axis 3) and then a column (axis 2).
constexpr int C32_PP = 4;
template <typename T>
__global__ void __launch_bounds__(128) k_fft_planes_c32(const c_t<T> *in, int f0, c_t<T> *work) {
    using C = c_t<T>;
    constexpr int N = 32, RS = N + 1;
    __shared__ __align__(16) C buf[C32_PP * N * RS];
    const int tid = threadIdx.x, q = tid >> 5, l = tid & 31;
    const size_t p0 = (size_t)blockIdx.x * C32_PP;   // first plane (field, k1) of the batch
    const C *src = in + ((size_t)f0 * N + p0) * N * N;
    for (int i = tid; i < C32_PP * N * N; i += 128) buf[(i >> 5) * RS + (i & 31)] = src[i];
    __syncthreads();
    C a[N];
    C *row = buf + (q * N + l) * RS;
#pragma unroll
    for (int j = 0; j < N; ++j) a[j] = row[j];
    RegFFT<T, N>::run(a);
#pragma unroll
    for (int j = 0; j < N; ++j) row[j] = a[j];
    __syncwarp();   // the plane's rows are complete (one warp per plane)
    C *col = buf + q * N * RS + l;
#pragma unroll
    for (int j = 0; j < N; ++j) a[j] = col[j * RS];
    RegFFT<T, N>::run(a);
#pragma unroll
    for (int j = 0; j < N; ++j) col[j * RS] = a[j];
    __syncthreads();
    C *dst = work + p0 * N * N;
    for (int i = tid; i < C32_PP * N * N; i += 128) dst[i] = buf[(i >> 5) * RS + (i & 31)];
}
// Columns: a thread transforms one axis-1 column (loads and stores coalesced across the warp) and
// writes Re(i^rot x) of the real field.
template <typename T>
__global__ void __launch_bounds__(256) k_fft_columns_re32(int f0, int nf, const c_t<T> *work, T *out,
                                                          const int4 *terms, int nT) {
    using C = c_t<T>;
    constexpr int N = 32, NC = N * N;
    const size_t gc = (size_t)blockIdx.x * 256 + threadIdx.x;
    const int fl = (int)(gc / NC), c = (int)(gc % NC);
    if (fl >= nf) return;
    const C *in = work + (size_t)fl * N * NC + c;
    C a[N];
#pragma unroll
    for (int r = 0; r < N; ++r) a[r] = in[(size_t)r * NC];
    RegFFT<T, N>::run(a);
    const int f = f0 + fl;
    const int rot = terms ? terms[f % nT].w : 0;
    T *o = out + (size_t)f * N * NC + c;
#pragma unroll
    for (int k = 0; k < N; ++k) o[(size_t)k * NC] = cipow(a[k], rot).x;
}

template <typename T>
void fft_complex_realpart(const Geometry &g, const c_t<T> *in, int f0, int nf, c_t<T> *work, T *out,
                          const c_t<T> *const W[3], const int4 *terms, int nT, cudaStream_t s) {
    using C = c_t<T>;
    if constexpr (sizeof(T) == 4) {
        if (g.n[0] == 32 && g.n[1] == 32 && g.n[2] == 32) {
            k_fft_planes_c32<T><<<(unsigned)((size_t)nf * 32 / C32_PP), 128, 0, s>>>(in, f0, work);
            k_fft_columns_re32<T><<<(unsigned)(((size_t)nf * 1024 + 255) / 256), 256, 0, s>>>(f0, nf, work, out,
                                                                                            terms, nT);
            count_launches(2);
            return;
        }
    }
    const size_t sm1 = (g.n[1] + g.n[2] + 2 * (size_t)g.n[1] * g.n[2]) * sizeof(C);
    if (sm1 > 48 * 1024)
        cudaFuncSetAttribute(k_fft_planes_c<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm1);
    k_fft_planes_c<T><<<(unsigned)((size_t)g.n[0] * nf), 256, sm1, s>>>(g, in, f0, work, W[1], W[2]);
    const int ncol = g.n[1] * g.n[2];
    int cb = (int)((48 * 1024 / sizeof(C) - g.n[0]) / (2 * g.n[0]));
    cb = std::max(1, std::min(cb, ncol));
    const size_t sm2 = (g.n[0] + 2 * (size_t)g.n[0] * cb) * sizeof(C);
    k_fft_columns_re<T><<<(unsigned)(((ncol + cb - 1) / cb) * (size_t)nf), 256, sm2, s>>>(g, f0, cb, work, out, W[0],
                                                                                          terms, nT);
    count_launches(2);
}

// phi_mu(G) = b f(|G|) exp(iG.r_mu) at voxel G (zone h, cell k), sorted site position s
template <typename T>
__device__ __forceinline__ c_t<T> site_amp(const RecombParams<T> &p, int s, const int h[3], const int k[3], T s2,
                                           int &cls, T &f) {
    if (s == 0 || s == p.ff.cls_end[cls]) {
        if (s > 0) ++cls;
        f = form_factor<T>(p.ff.cls_kind[cls], p.ff.cls_coef[cls], s2);
    }
    const int site = p.site_of[s];
    const c_t<T> *tH = p.phH + (size_t)site * 3 * p.nHmax;
    const c_t<T> *tk = p.phk + (size_t)site * 3 * p.nmax;
    c_t<T> ph = cmul(cmul(tH[h[0]], tH[p.nHmax + h[1]]), tH[2 * p.nHmax + h[2]]);
    ph = cmul(ph, cmul(cmul(tk[k[0]], tk[p.nmax + k[1]]), tk[2 * p.nmax + k[2]]));
    return cscale(ph, f * p.scat[site]);
}

constexpr int ADJ_ZC = 32;  // zones staged per chunk

// acc += c b for a real c and a complex b: one paired FMA (FFMA2) in FP32
__device__ __forceinline__ void acc_cb(float2 &acc, float c, float2 b) {
    acc = __ffma2_rn(make_float2(c, c), b, acc);
}
__device__ __forceinline__ void acc_cb(double2 &acc, double c, double2 b) {
    acc.x = fma(c, b.x, acc.x);
    acc.y = fma(c, b.y, acc.y);
}

// Z_{m,mu,t}(k) for the displacive path; sorted site positions, full k index.  MAXS: sites held
// per thread (exact site count up to 8)
template <typename T, int MAXS, int TPT>
__global__ void __launch_bounds__(256) k_adj_z_disp(const __grid_constant__ RecombParams<T> p, const T *dLdI,
                                                   const c_t<T> *F, int P, double scale, c_t<T> *Z) {
    using C = c_t<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *beta = (C *)smem_raw;                               // [ZC][nsite]
    T *pw = (T *)(beta + (size_t)ADJ_ZC * p.nsite);        // [ZC][3][P+1]
    const Geometry &g = p.g;
    const GridMap &gm = p.gm;
    const int k = blockIdx.x;
    const int kk[3] = {k / (g.n[1] * g.n[2]), (k / g.n[2]) % g.n[1], k % g.n[2]};
    int lo[3], nz[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        lo[a] = -fdiv(-(gm.g0[a] - kk[a]), g.n[a]);
        const int hi = fdiv(gm.g0[a] + gm.cnt[a] - 1 - kk[a], g.n[a]);
        nz[a] = max(0, hi - lo[a] + 1);
    }
    const int nzk = nz[0] * nz[1] * nz[2];
    const size_t nv = (size_t)gm.cnt[0] * gm.cnt[1] * gm.cnt[2];
    int tt[TPT];
    int4 e[TPT];
#pragma unroll
    for (int j = 0; j < TPT; ++j) {
        tt[j] = blockIdx.y * (256 * TPT) + threadIdx.x + 256 * j;
        e[j] = tt[j] < p.nT ? p.terms[tt[j]] : make_int4(0, 0, 0, 0);
    }
    C acc[TPT][MAXS];
#pragma unroll
    for (int j = 0; j < TPT; ++j)
#pragma unroll
        for (int s = 0; s < MAXS; ++s) acc[j][s] = mk<T>(T(0), T(0));

    for (int z0 = 0; z0 < nzk; z0 += ADJ_ZC) {
        const int zc = min(ADJ_ZC, nzk - z0);
        __syncthreads();
        // stage: scaled Q powers and beta_mu = scale dL/dI conj(F) phi_mu for each zone
        for (int idx = threadIdx.x; idx < zc * 4; idx += blockDim.x) {
            const int zi = idx >> 2, part = idx & 3;
            const int z = z0 + zi;
            const int i1 = z / (nz[1] * nz[2]), i2 = (z / nz[2]) % nz[1], i3 = z % nz[2];
            const int G[3] = {g.n[0] * (lo[0] + i1) + kk[0], g.n[1] * (lo[1] + i2) + kk[1], g.n[2] * (lo[2] + i3) + kk[2]};
            double Qd[3];
#pragma unroll
            for (int a = 0; a < 3; ++a)
                Qd[a] = (double)G[0] / g.n[0] * p.recip[a] + (double)G[1] / g.n[1] * p.recip[3 + a] +
                        (double)G[2] / g.n[2] * p.recip[6 + a];
            if (part < 3) {
                const T qs = (T)((double)G[part] / g.n[part] / p.gscale[part]);  // x_part, |x| <= 1
                T *dst = pw + ((size_t)zi * 3 + part) * (P + 1);
                T v = T(1);
                for (int q = 0; q <= P; ++q) {
                    dst[q] = v;
                    v *= qs;
                }
            } else {
                const size_t vox = ((size_t)(G[0] - gm.g0[0]) * gm.cnt[1] + (G[1] - gm.g0[1])) * gm.cnt[2] + (G[2] - gm.g0[2]);
                const C Fv = F[(size_t)p.model * nv + vox];
                const T gI = dLdI[vox] * (T)scale;
                const C gam = mk<T>(gI * Fv.x, -gI * Fv.y);
                const T s2 = (T)((Qd[0] * Qd[0] + Qd[1] * Qd[1] + Qd[2] * Qd[2]) / (FOUR_PI_D * FOUR_PI_D));
                const int h[3] = {lo[0] + i1 - gm.Hmin[0], lo[1] + i2 - gm.Hmin[1], lo[2] + i3 - gm.Hmin[2]};
                int cls = 0;
                T f = T(1);
                for (int s = 0; s < p.nsite; ++s) beta[(size_t)zi * p.nsite + s] = cmul(gam, site_amp<T>(p, s, h, kk, s2, cls, f));
            }
        }
        __syncthreads();
        for (int zi = 0; zi < zc; ++zi) {
            const T *pz = pw + (size_t)zi * 3 * (P + 1);
            T c[TPT];
#pragma unroll
            for (int j = 0; j < TPT; ++j) c[j] = pz[e[j].x] * pz[(P + 1) + e[j].y] * pz[2 * (P + 1) + e[j].z];
#pragma unroll
            for (int s = 0; s < MAXS; ++s) {
                if (s < p.nsite) {
                    const C b = beta[(size_t)zi * p.nsite + s];
#pragma unroll
                    for (int j = 0; j < TPT; ++j) acc_cb(acc[j][s], c[j], b);
                }
            }
        }
    }
#pragma unroll
    for (int j = 0; j < TPT; ++j) {
        if (tt[j] >= p.nT) continue;
#pragma unroll
        for (int s = 0; s < MAXS; ++s)
            if (s < p.nsite) {
                const int site = p.site_of[s];
                Z[(((size_t)p.model * p.nsite + site) * p.nT + tt[j]) * g.ncell + k] = acc[j][s];
            }
    }
}

// Z_{m,mu,alpha}(k) for the magnetic path: one thread per (site, component) of one k
template <typename T>
__global__ void k_adj_z_mag(const __grid_constant__ RecombParams<T> p, const T *dLdI, const c_t<T> *F, double scale,
                            c_t<T> *Z) {
    using C = c_t<T>;
    const Geometry &g = p.g;
    const GridMap &gm = p.gm;
    const int k = blockIdx.x;
    const int kk[3] = {k / (g.n[1] * g.n[2]), (k / g.n[2]) % g.n[1], k % g.n[2]};
    const int s = threadIdx.x / 3, alpha = threadIdx.x % 3;
    if (s >= p.nsite) return;
    int lo[3], nz[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        lo[a] = -fdiv(-(gm.g0[a] - kk[a]), g.n[a]);
        const int hi = fdiv(gm.g0[a] + gm.cnt[a] - 1 - kk[a], g.n[a]);
        nz[a] = max(0, hi - lo[a] + 1);
    }
    const size_t nv = (size_t)gm.cnt[0] * gm.cnt[1] * gm.cnt[2];
    C acc = mk<T>(T(0), T(0));
    for (int z = 0; z < nz[0] * nz[1] * nz[2]; ++z) {
        const int i1 = z / (nz[1] * nz[2]), i2 = (z / nz[2]) % nz[1], i3 = z % nz[2];
        const int G[3] = {g.n[0] * (lo[0] + i1) + kk[0], g.n[1] * (lo[1] + i2) + kk[1], g.n[2] * (lo[2] + i3) + kk[2]};
        double Qd[3];
#pragma unroll
        for (int a = 0; a < 3; ++a)
            Qd[a] = (double)G[0] / g.n[0] * p.recip[a] + (double)G[1] / g.n[1] * p.recip[3 + a] +
                    (double)G[2] / g.n[2] * p.recip[6 + a];
        const double q2 = Qd[0] * Qd[0] + Qd[1] * Qd[1] + Qd[2] * Qd[2];
        const size_t vox = ((size_t)(G[0] - gm.g0[0]) * gm.cnt[1] + (G[1] - gm.g0[1])) * gm.cnt[2] + (G[2] - gm.g0[2]);
        const C *Fv = F + ((size_t)p.model * nv + vox) * 3;
        C PF;
        if (q2 > 0) {
            const T qa = (T)(Qd[alpha] / sqrt(q2));
            C dot = mk<T>(T(0), T(0));
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                const T qb = (T)(Qd[b] / sqrt(q2));
                dot.x += qb * Fv[b].x;
                dot.y += qb * Fv[b].y;
            }
            PF = mk<T>(Fv[alpha].x - qa * dot.x, Fv[alpha].y - qa * dot.y);
        } else {
            PF = cscale(Fv[alpha], T(2) / T(3));
        }
        const T gI = dLdI[vox] * (T)scale;
        const C gam = mk<T>(gI * PF.x, -gI * PF.y);
        const int h[3] = {lo[0] + i1 - gm.Hmin[0], lo[1] + i2 - gm.Hmin[1], lo[2] + i3 - gm.Hmin[2]};
        // class of sorted position s: walk the class ends
        int cls = 0;
        while (s >= p.ff.cls_end[cls]) ++cls;
        const T s2 = (T)(q2 / (FOUR_PI_D * FOUR_PI_D));
        const T f = form_factor<T>(p.ff.cls_kind[cls], p.ff.cls_coef[cls], s2);
        const int site = p.site_of[s];
        const C *tH = p.phH + (size_t)site * 3 * p.nHmax;
        const C *tk = p.phk + (size_t)site * 3 * p.nmax;
        C ph = cmul(cmul(tH[h[0]], tH[p.nHmax + h[1]]), tH[2 * p.nHmax + h[2]]);
        ph = cmul(ph, cmul(cmul(tk[kk[0]], tk[p.nmax + kk[1]]), tk[2 * p.nmax + kk[2]]));
        acc = cadd(acc, cmul(gam, cscale(ph, f * p.scat[site])));
    }
    const int site = p.site_of[s];
    Z[(((size_t)p.model * p.nsite + site) * 3 + alpha) * g.ncell + k] = acc;
}

// grad[m][mu][cell][alpha] = sum_j gs_j b*_{j,alpha} w sum_t D_t(cell) field_{t - e_j}(cell) / w
struct GradAxes {
    double bg[9];  // gs_j b*_{j,alpha}, row j
};

template <typename T>
__global__ void k_adj_gather(int nmodels, int nsite, int ncell, int P, int nT, const int4 *terms, const T *pw,
                             const uint8_t *occ, const T *D, const GradAxes ax, T *grad) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t natom = (size_t)nmodels * nsite * ncell;
    if (idx >= natom) return;
    const size_t ms = idx / ncell, cell = idx - ms * ncell;
    const size_t P1 = (size_t)P + 1;
    const T *px = pw + (ms * 3 + 0) * P1 * ncell + cell;
    const T *py = pw + (ms * 3 + 1) * P1 * ncell + cell;
    const T *pz = pw + (ms * 3 + 2) * P1 * ncell + cell;
    const T *d = D + ms * (size_t)nT * ncell + cell;
    T gx = T(0), gy = T(0), gz = T(0);
    for (int t = 0; t < nT; ++t) {
        const int4 e = terms[t];
        const T dv = d[(size_t)t * ncell];
        const T ax = px[(size_t)e.x * ncell], by = py[(size_t)e.y * ncell], cz = pz[(size_t)e.z * ncell];
        if (e.x > 0) gx = fma(dv, px[(size_t)(e.x - 1) * ncell] * by * cz, gx);
        if (e.y > 0) gy = fma(dv, ax * py[(size_t)(e.y - 1) * ncell] * cz, gy);
        if (e.z > 0) gz = fma(dv, ax * by * pz[(size_t)(e.z - 1) * ncell], gz);
    }
    const T w = occ ? (T)occ[idx] : T(1);
#pragma unroll
    for (int a = 0; a < 3; ++a)
        grad[idx * 3 + a] = w * ((T)ax.bg[a] * gx + (T)ax.bg[3 + a] * gy + (T)ax.bg[6 + a] * gz);
}

template <typename T>
__global__ void k_mag_grad_layout(int nmodels, int nsite, int ncell, const T *D, T *grad) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t tot = (size_t)nmodels * nsite * ncell * 3;
    if (idx >= tot) return;
    const int a = (int)(idx % 3);
    const size_t atom = idx / 3;
    const size_t ms = atom / ncell, cell = atom - ms * ncell;
    grad[idx] = D[(ms * 3 + a) * ncell + cell];
}

template <typename T>
ds_status backward_run(ds_model *M, const ds_qgrid *q, const ds_opts *o, const T *dLdI, T *grad, cudaStream_t st,
                       Scratch &ws) {
    using C = c_t<T>;
    ds_ctx *ctx = M->ctx;
    int g0[3], cnt[3];
    ds_status rc = grid_indices(ctx, M, q, g0, cnt);
    if (rc != DS_OK) return rc;
    const size_t nv = (size_t)cnt[0] * cnt[1] * cnt[2];
    const int nsite = M->nsite, nmod = M->nmodels;
    const bool mag = o->disorder == DS_SPIN;
    const int NC = mag ? 3 : 1;
    T *Ifwd = (T *)ws.get(sizeof(T) * nv);
    C *F = (C *)ws.get(sizeof(C) * nv * nmod * NC);
    if (ws.failed) return ds_fail(ctx, DS_ERR_OOM, "device allocation failed (adjoint)");
    ForwardKeep<T> keep;
    keep.Fout = F;
    ds_result_info info;
    memset(&info, 0, sizeof(info));
    rc = plan_and_run<T>(M, q, o, Ifwd, st, ws, &info, &keep);
    if (rc != DS_OK) return rc;
    RecombParams<T> p = keep.p;
    const Geometry &g = keep.g;
    const double N = (double)nsite * g.ncell;
    const int nT = mag ? 3 : p.nT;
    const size_t nfield = (size_t)nmod * nsite * nT;
    C *Z = (C *)ws.get(sizeof(C) * nfield * g.ncell);
    T *D = (T *)ws.get(sizeof(T) * nfield * g.ncell);
    const int fb = (int)std::max<size_t>(1, std::min<size_t>(nfield, (256ull << 20) / (sizeof(C) * (size_t)g.ncell)));
    C *work = (C *)ws.get(sizeof(C) * (size_t)fb * g.ncell);
    if (ws.failed) return ds_fail(ctx, DS_ERR_OOM, "device allocation failed (adjoint spectra)");
    if (ws.total > ctx->budget)
        return ds_fail(ctx, DS_ERR_ADMISSION, "adjoint needs %zu bytes of scratch, budget %zu", ws.total, ctx->budget);
    {
        ProfScope ps(ctx, "adjoint_z", st);
        for (int m = 0; m < nmod; ++m) {
            p.model = m;
            bool done = false;
            if constexpr (sizeof(T) == 4) {
                // FP32: the transposed sum factorisation over each k's zones (adjoint_sf.cu)
                if (!mag) done = adjoint_z_disp_sf(p, dLdI, F, keep.src.P, 2.0 / (nmod * N), Z, st);
            }
            if (done) {
            } else if (mag) {
                k_adj_z_mag<T><<<g.ncell, 3 * nsite, 0, st>>>(p, dLdI, F, 2.0 * 0.07265 / (nmod * N), Z);
            } else {
                constexpr int TPT = sizeof(T) == 4 ? 4 : 2;
                const size_t sm = (size_t)ADJ_ZC * nsite * sizeof(C) + (size_t)ADJ_ZC * 3 * (keep.src.P + 1) * sizeof(T);
                auto launch = [&](auto kern, int tpt) {
                    if (sm > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
                    dim3 gr(g.ncell, (nT + 256 * tpt - 1) / (256 * tpt));
                    kern<<<gr, 256, sm, st>>>(p, dLdI, F, keep.src.P, 2.0 / (nmod * N), Z);
                };
                switch (nsite) {
                    case 1: launch(k_adj_z_disp<T, 1, TPT>, TPT); break;
                    case 2: launch(k_adj_z_disp<T, 2, TPT>, TPT); break;
                    case 3: launch(k_adj_z_disp<T, 3, TPT>, TPT); break;
                    case 4: launch(k_adj_z_disp<T, 4, TPT>, TPT); break;
                    case 5: launch(k_adj_z_disp<T, 5, TPT>, TPT); break;
                    case 6: launch(k_adj_z_disp<T, 6, TPT>, TPT); break;
                    case 7: launch(k_adj_z_disp<T, 7, TPT>, TPT); break;
                    case 8: launch(k_adj_z_disp<T, 8, TPT>, TPT); break;
                    default: launch(k_adj_z_disp<T, 16, 1>, 1); break;
                }
            }
            if (!done) count_launches(1);
        }
    }
    {
        ProfScope ps(ctx, "adjoint_fft", st);
        for (size_t f0 = 0; f0 < nfield; f0 += fb)
            fft_complex_realpart<T>(g, Z, (int)f0, (int)std::min<size_t>(fb, nfield - f0), work, D, keep.W,
                                    mag ? nullptr : keep.terms, nT, st);
    }
    {
        ProfScope ps(ctx, "adjoint_gather", st);
        const size_t natom = (size_t)nmod * nsite * g.ncell;
        if (mag) {
            k_mag_grad_layout<T><<<(unsigned)((natom * 3 + 255) / 256), 256, 0, st>>>(nmod, nsite, g.ncell, D, grad);
        } else {
            GradAxes ax;
            for (int j = 0; j < 3; ++j)
                for (int a = 0; a < 3; ++a) ax.bg[3 * j + a] = p.gscale[j] * p.recip[3 * j + a];
            k_adj_gather<T><<<(unsigned)((natom + 255) / 256), 256, 0, st>>>(
                nmod, nsite, g.ncell, keep.src.P, nT, keep.terms, keep.pw, M->has_occ ? M->d_occ : nullptr, D,
                ax, grad);
        }
        count_launches(1);
    }
    if (cudaGetLastError() != cudaSuccess) return ds_fail(ctx, DS_ERR_CUDA, "adjoint launch failed");
    return DS_OK;
}

template <typename T>
ds_status backward_entry(ds_model *M, const ds_qgrid *q, const ds_opts *o, const void *dLdI, void *grad, int dev,
                         cudaStream_t st) {
    ds_ctx *ctx = M->ctx;
    int g0[3], cnt[3];
    ds_status rc = grid_indices(ctx, M, q, g0, cnt);
    if (rc != DS_OK) return rc;
    const size_t nv = (size_t)cnt[0] * cnt[1] * cnt[2];
    const size_t ng = (size_t)M->nmodels * M->nsite * M->n[0] * M->n[1] * M->n[2] * 3;
    Scratch ws(st);
    const T *d_in = (const T *)dLdI;
    T *d_grad = (T *)grad;
    if (!dev) {
        T *a = (T *)ws.get(sizeof(T) * nv);
        d_grad = (T *)ws.get(sizeof(T) * ng);
        if (ws.failed) return ds_fail(ctx, DS_ERR_OOM, "device allocation failed");
        if (cudaMemcpyAsync(a, dLdI, sizeof(T) * nv, cudaMemcpyHostToDevice, st) != cudaSuccess)
            return ds_fail(ctx, DS_ERR_CUDA, "copy of dL/dI failed");
        d_in = a;
    }
    rc = backward_run<T>(M, q, o, d_in, d_grad, st, ws);
    if (rc == DS_OK && !dev) {
        if (cudaMemcpyAsync(grad, d_grad, sizeof(T) * ng, cudaMemcpyDeviceToHost, st) != cudaSuccess)
            rc = ds_fail(ctx, DS_ERR_CUDA, "copy of the gradient failed");
    }
    ws.release();
    if (!dev || rc != DS_OK) cudaStreamSynchronize(st);
    return rc;
}

}  // namespace

extern "C" ds_status ds_backward(ds_model *M, const ds_qgrid *q, const ds_opts *o, const void *dLdI, void *grad,
                                 int is_device, void *stream) {
    if (!M) return DS_ERR_ARG;
    ds_ctx *ctx = M->ctx;
    if (!dLdI || !grad) return ds_fail(ctx, DS_ERR_ARG, "null buffer");
    ds_status rc = check_request(M, q, o);
    if (rc != DS_OK) return rc;
    if (o->disorder == DS_OCC) return ds_fail(ctx, DS_ERR_UNSUPPORTED, "occupancies are discrete: no gradient");
    if (o->mode != DS_TOTAL) return ds_fail(ctx, DS_ERR_UNSUPPORTED, "the adjoint is defined for DS_TOTAL mode");
    if (o->smoothing != DS_SMOOTH_NONE) return ds_fail(ctx, DS_ERR_UNSUPPORTED, "the adjoint takes no smoothing");
    if (o->taylor_zonal) return ds_fail(ctx, DS_ERR_UNSUPPORTED, "the adjoint uses one Taylor order for the grid");
    if (o->dw_coupling) return ds_fail(ctx, DS_ERR_UNSUPPORTED, "the adjoint does not differentiate the Debye-Waller coupling");
    if (cudaSetDevice(ctx->device) != cudaSuccess) return ds_fail(ctx, DS_ERR_CUDA, "cudaSetDevice");
    cudaStream_t st = (cudaStream_t)stream;
    if (o->precision == DS_FP64) return backward_entry<double>(M, q, o, dLdI, grad, is_device, st);
    return backward_entry<float>(M, q, o, dLdI, grad, is_device, st);
}
