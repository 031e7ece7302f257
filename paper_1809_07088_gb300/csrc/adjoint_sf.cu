// Transposed sum factorisation for the displacive adjoint (FP32; the chain rule of Section III C,
// TOTAL mode, no counterpart in the paper).
//
// For one k and one site, the adjoint of the Taylor recombination needs
//     Z_abc(k) = sum_{H: H + k in grid} x1^a x2^b x3^c beta(H),
//     beta(H) = scale dL/dI(G) conj(F(G)) b f(|G|) exp(iG.r_mu),  x_j = g_j / gs_j,
// the transpose of the forward polynomial evaluation over the zones of k.  It separates along the
// grid axes like the forward (taylor_sf.cu), now as three power sums:
//     W[a](h2, h3) = sum_h1 x1(h1)^a beta(h1, h2, h3)
//     V[a, b](h3)  = sum_h2 x2(h2)^b W[a](h2, h3)
//     Z[a, b, c]   = sum_h3 x3(h3)^c V[a, b](h3)
// with the powers of each axis tabulated once per k.  Each thread owns one output row of a step and
// four consecutive powers (registers); every sum runs over the zones of one axis in a fixed order.
//
// CTA: one k of the full grid (the adjoint's complex FFT takes every k), shared memory sized for the
// widest zone box of the grid (zr zones per axis), 128, 256 or 512 threads as that footprint lets
// 16 warps reside on an SM; per site the
// zone factors beta are formed from gamma = scale dL/dI conj(F) (shared memory, once per k) and the
// site's phases and form factor.
#include <algorithm>
#include <cmath>

#include "internal.h"

namespace ds {

namespace {

constexpr int AS_ZR = 17;        // zones per axis handled (at most)
constexpr int AS_PMAX = 31;      // Taylor order handled
constexpr int AS_CH = 4;         // powers per thread item (one 16-byte load of the power table)

__host__ __device__ __forceinline__ int fdivf(int a, int b) {
    int q = a / b;
    if ((a % b != 0) && ((a < 0) != (b < 0))) --q;
    return q;
}

// x / d for 0 <= x < 2^16 and 1 <= d < 2^15 as a multiply-high by m = ceil(2^32 / d): with
// m d = 2^32 + e, 0 <= e < d, and x = q d + r, floor(x m / 2^32) = q + floor((r + x e / 2^32) / d) = q
// because x e < 2^32 (d = 1 takes m = 0 and x itself)
struct ItemDiv {
    int d;
    unsigned m;
    __device__ __forceinline__ explicit ItemDiv(int dd) : d(dd), m(dd == 1 ? 0u : 0xFFFFFFFFu / (unsigned)dd + 1u) {}
    __device__ __forceinline__ int div(int x) const { return m ? (int)__umulhi((unsigned)x, m) : x; }
};

struct AdjLayout {
    size_t gam, bv, W, pw, total;
};
__host__ __device__ __forceinline__ AdjLayout adj_layout(int P, int zr) {
    auto al = [](size_t x) { return (x + 15) & ~(size_t)15; };
    const size_t z3 = (size_t)zr * zr * zr, nab = (size_t)(P + 1) * (P + 2) / 2;
    AdjLayout L;
    L.gam = 0;
    L.bv = al(L.gam + z3 * sizeof(float2));
    L.W = al(L.bv + std::max(z3, nab * zr) * sizeof(float2));
    L.pw = al(L.W + (size_t)(P + 1) * zr * zr * sizeof(float2));
    L.total = al(L.pw + (size_t)3 * zr * ((P + 1 + 3) & ~3) * sizeof(float));   // rows padded to 4
    return L;
}

}  // namespace

template <int AS_THREADS>
__global__ void __launch_bounds__(AS_THREADS, 512 / AS_THREADS)
    k_adj_taylor_sf(const __grid_constant__ RecombParams<float> p, const float *dLdI, const float2 *F, int P, int zr,
                    float scale, float2 *Z) {
    extern __shared__ __align__(16) unsigned char smem[];
    const Geometry &g = p.g;
    const GridMap &gm = p.gm;
    const int k = blockIdx.x;
    const int n1 = g.n[0], n2 = g.n[1], n3 = g.n[2];
    const int kk[3] = {k / (n2 * n3), (k / n3) % n2, k % n3};
    int lo[3], nz[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        lo[a] = -fdivf(-(gm.g0[a] - kk[a]), g.n[a]);
        const int hi = fdivf(gm.g0[a] + gm.cnt[a] - 1 - kk[a], g.n[a]);
        nz[a] = max(0, hi - lo[a] + 1);
    }
    const int nsite = p.nsite, nT = p.nT, P1 = P + 1, P1p = (P1 + 3) & ~3;   // power rows padded to 4
    const int tid = threadIdx.x;
    const size_t ncell = g.ncell;
    if (nz[0] * nz[1] * nz[2] == 0) {
        // no voxel of the grid has this k: every Z(k) is zero
        for (int i = tid; i < nsite * nT; i += AS_THREADS) {
            const int s = i / nT, t = i - s * nT;
            Z[(((size_t)p.model * nsite + s) * nT + t) * ncell + k] = make_float2(0.f, 0.f);
        }
        return;
    }
    const int nz1 = nz[0], nz2 = nz[1], nz3 = nz[2], ncol = nz2 * nz3, nzone = nz1 * ncol;
    const ItemDiv dcol(ncol), dz3(nz3), dch((P + 1 + AS_CH - 1) / AS_CH);
    const AdjLayout L = adj_layout(P, zr);
    float2 *gam = (float2 *)(smem + L.gam);   // [h1][h2][h3]
    float2 *bv = (float2 *)(smem + L.bv);     // beta [h1][col], then V [(a, b)][h3]
    float2 *W = (float2 *)(smem + L.W);       // [a][col]
    float *pw = (float *)(smem + L.pw);       // [axis][zone][e]

    // powers x_a(j)^e of the scaled coefficient variables
    for (int i = tid; i < 3 * zr; i += AS_THREADS) {
        const int a = i / zr, j = i - a * zr;
        const double x = ((double)(lo[a] + j) + (double)kk[a] / g.n[a]) / p.gscale[a];
        double v = 1.0;
        for (int e = 0; e <= P; ++e) {
            pw[(size_t)i * P1p + e] = j < nz[a] ? (float)v : 0.f;
            v *= x;
        }
        for (int e = P1; e < P1p; ++e) pw[(size_t)i * P1p + e] = 0.f;
    }
    // gamma = scale dL/dI conj(F) of the model, per zone of the box
    const size_t nv = (size_t)gm.cnt[0] * gm.cnt[1] * gm.cnt[2];
    for (int z = tid; z < nzone; z += AS_THREADS) {
        const int j = z / ncol, col = z - j * ncol, h2 = col / nz3, h3 = col - h2 * nz3;
        const int G1 = n1 * (lo[0] + j) + kk[0], G2 = n2 * (lo[1] + h2) + kk[1], G3 = n3 * (lo[2] + h3) + kk[2];
        const size_t v = ((size_t)(G1 - gm.g0[0]) * gm.cnt[1] + (G2 - gm.g0[1])) * gm.cnt[2] + (G3 - gm.g0[2]);
        const float2 Fv = F[(size_t)p.model * nv + v];
        float gI = dLdI[v] * scale;
        if (p.ff.ncls == 1) {
            // one form-factor class: f(|G|) enters every beta of the zone, folded in here once
            float Q[3];
#pragma unroll
            for (int a = 0; a < 3; ++a)
                Q[a] = fmaf((float)G1, p.qstep[a], fmaf((float)G2, p.qstep[3 + a], (float)G3 * p.qstep[6 + a]));
            const float q2 = Q[0] * Q[0] + Q[1] * Q[1] + Q[2] * Q[2];
            float f = p.ff.cls_gc[0];
            for (int i = 0; i < p.ff.cls_ng[0]; ++i) f = fmaf(p.ff.cls_ga[0][i], exp2_w(p.ff.cls_gb[0][i] * q2), f);
            gI *= f;
        }
        gam[z] = make_float2(gI * Fv.x, -gI * Fv.y);
    }
    __syncthreads();

    const int nab = P1 * (P1 + 1) / 2;
    int cls = 0;
    for (int s = 0; s < nsite; ++s) {
        if (s == p.ff.cls_end[cls]) ++cls;
        const int site = p.site_of[s];
        // beta = gamma b f(|G|) exp(iG.r_mu)
        {
            const c_t<float> *tH = p.phH + (size_t)site * 3 * p.nHmax;
            const c_t<float> *tk = p.phk + (size_t)site * 3 * p.nmax;
            const float2 pk = cscale(cmul(cmul(tk[kk[0]], tk[p.nmax + kk[1]]), tk[2 * p.nmax + kk[2]]), p.scat[site]);
            for (int z = tid; z < nzone; z += AS_THREADS) {
                const int j = z / ncol, col = z - j * ncol, h2 = col / nz3, h3 = col - h2 * nz3;
                float f = 1.f;
                if (p.ff.ncls != 1) {
                    const int G1 = n1 * (lo[0] + j) + kk[0], G2 = n2 * (lo[1] + h2) + kk[1], G3 = n3 * (lo[2] + h3) + kk[2];
                    float Q[3];
#pragma unroll
                    for (int a = 0; a < 3; ++a)
                        Q[a] = fmaf((float)G1, p.qstep[a], fmaf((float)G2, p.qstep[3 + a], (float)G3 * p.qstep[6 + a]));
                    const float q2 = Q[0] * Q[0] + Q[1] * Q[1] + Q[2] * Q[2];
                    f = p.ff.cls_gc[cls];
                    for (int i = 0; i < p.ff.cls_ng[cls]; ++i) f = fmaf(p.ff.cls_ga[cls][i], exp2_w(p.ff.cls_gb[cls][i] * q2), f);
                }
                const float2 ph = cmul(cmul(tH[lo[0] + j - gm.Hmin[0]], tH[p.nHmax + lo[1] + h2 - gm.Hmin[1]]),
                                       tH[2 * p.nHmax + lo[2] + h3 - gm.Hmin[2]]);
                bv[z] = cmul(gam[z], cscale(cmul(ph, pk), f));
            }
        }
        __syncthreads();
        // W[a][col] = sum_h1 x1(h1)^a beta(h1, col), four powers per item
        const int nch = (P1 + AS_CH - 1) / AS_CH;
        for (int it = tid; it < ncol * nch; it += AS_THREADS) {
            const int ch = dcol.div(it), col = it - ch * ncol, a0 = ch * AS_CH;
            float2 acc[AS_CH];
#pragma unroll
            for (int q = 0; q < AS_CH; ++q) acc[q] = make_float2(0.f, 0.f);
            for (int h1 = 0; h1 < nz1; ++h1) {
                const float2 b = bv[h1 * ncol + col];
                const float4 p4 = *(const float4 *)(pw + (size_t)(0 * zr + h1) * P1p + a0);
                const float pp[AS_CH] = {p4.x, p4.y, p4.z, p4.w};
#pragma unroll
                for (int q = 0; q < AS_CH; ++q)
                    if (a0 + q < P1) acc[q] = __ffma2_rn(make_float2(pp[q], pp[q]), b, acc[q]);
            }
#pragma unroll
            for (int q = 0; q < AS_CH; ++q)
                if (a0 + q < P1) W[(size_t)(a0 + q) * ncol + col] = acc[q];
        }
        __syncthreads();
        // V[(a, b)][h3] = sum_h2 x2(h2)^b W[a](h2, h3), b <= P - a, four powers per item
        for (int it = tid; it < P1 * nch * nz3; it += AS_THREADS) {
            const int r = dz3.div(it), h3 = it - r * nz3, a = dch.div(r), b0 = (r - a * nch) * AS_CH;
            if (b0 > P - a) continue;
            float2 acc[AS_CH];
#pragma unroll
            for (int q = 0; q < AS_CH; ++q) acc[q] = make_float2(0.f, 0.f);
            for (int h2 = 0; h2 < nz2; ++h2) {
                const float2 w = W[(size_t)a * ncol + h2 * nz3 + h3];
                const float4 p4 = *(const float4 *)(pw + (size_t)(1 * zr + h2) * P1p + b0);
                const float pp[AS_CH] = {p4.x, p4.y, p4.z, p4.w};
#pragma unroll
                for (int q = 0; q < AS_CH; ++q)
                    if (b0 + q <= P - a) acc[q] = __ffma2_rn(make_float2(pp[q], pp[q]), w, acc[q]);
            }
            const int ab0 = a * P1 - a * (a - 1) / 2;   // pairs (a', b') with a' < a
#pragma unroll
            for (int q = 0; q < AS_CH; ++q)
                if (b0 + q <= P - a) bv[(size_t)(ab0 + b0 + q) * nz3 + h3] = acc[q];
        }
        __syncthreads();
        // Z[t(a, b, c)](k) = sum_h3 x3(h3)^c V[(a, b)](h3), c <= P - a - b, four powers per item
        float2 *Zs = Z + (((size_t)p.model * nsite + site) * nT) * ncell + k;
        for (int it = tid; it < nab * nch; it += AS_THREADS) {
            const int ab = dch.div(it), c0 = (it - ab * nch) * AS_CH;
            // (a, b) of pair index ab: a is the largest with ab0(a) = a (2 P1 - a + 1) / 2 <= ab, the
            // smaller root of the quadratic (FP32 square root, one integer correction each way)
            const float Bq = (float)(2 * P1 + 1);
            int a = min((int)(0.5f * (Bq - sqrtf(fmaxf(0.f, Bq * Bq - 8.f * (float)ab)))), P);
            if (a * (2 * P1 - a + 1) / 2 > ab) --a;
            if (a < P && (a + 1) * (2 * P1 - a) / 2 <= ab) ++a;
            const int b = ab - a * (2 * P1 - a + 1) / 2;
            const int lc = P - a - b;
            if (c0 > lc) continue;
            float2 acc[AS_CH];
#pragma unroll
            for (int q = 0; q < AS_CH; ++q) acc[q] = make_float2(0.f, 0.f);
            for (int h3 = 0; h3 < nz3; ++h3) {
                const float2 v = bv[(size_t)ab * nz3 + h3];
                const float4 p4 = *(const float4 *)(pw + (size_t)(2 * zr + h3) * P1p + c0);
                const float pp[AS_CH] = {p4.x, p4.y, p4.z, p4.w};
#pragma unroll
                for (int q = 0; q < AS_CH; ++q)
                    if (c0 + q <= lc) acc[q] = __ffma2_rn(make_float2(pp[q], pp[q]), v, acc[q]);
            }
            // monomial index of (a, b, c): lexicographic order, a outer, b middle, c inner; the
            // monomials with a' < a number T(P) - T(P - a)
            const int t0 = (P1 * (P1 + 1) * (P1 + 2) - (P1 - a) * (P1 - a + 1) * (P1 - a + 2)) / 6 +
                           b * (P - a + 1) - b * (b - 1) / 2;
#pragma unroll
            for (int q = 0; q < AS_CH; ++q)
                if (c0 + q <= lc) Zs[(size_t)(t0 + c0 + q) * ncell] = acc[q];
        }
        __syncthreads();
    }
}

bool adjoint_z_disp_sf(const RecombParams<float> &p, const float *dLdI, const float2 *F, int P, double scale,
                       float2 *Z, cudaStream_t s) {
    if (P > AS_PMAX) return false;
    // widest zone box of any k along any axis
    int zr = 1;
    for (int a = 0; a < 3; ++a)
        for (int k = 0; k < p.g.n[a]; ++k) {
            const int lo = -fdivf(-(p.gm.g0[a] - k), p.g.n[a]);
            const int hi = fdivf(p.gm.g0[a] + p.gm.cnt[a] - 1 - k, p.g.n[a]);
            zr = std::max(zr, hi - lo + 1);
        }
    if (zr > AS_ZR) return false;
    const AdjLayout L = adj_layout(P, zr);
    if (L.total > 227 * 1024) return false;
    const unsigned nb = (unsigned)p.g.ncell;
    switch (sf_threads_for(L.total)) {
        case 128:
            cudaFuncSetAttribute(k_adj_taylor_sf<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.total);
            k_adj_taylor_sf<128><<<nb, 128, L.total, s>>>(p, dLdI, F, P, zr, (float)scale, Z);
            break;
        case 256:
            cudaFuncSetAttribute(k_adj_taylor_sf<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.total);
            k_adj_taylor_sf<256><<<nb, 256, L.total, s>>>(p, dLdI, F, P, zr, (float)scale, Z);
            break;
        default:
            cudaFuncSetAttribute(k_adj_taylor_sf<512>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.total);
            k_adj_taylor_sf<512><<<nb, 512, L.total, s>>>(p, dLdI, F, P, zr, (float)scale, Z);
            break;
    }
    count_launches(1);
    return true;
}

}  // namespace ds
