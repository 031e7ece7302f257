// Displacive (Taylor) recombination by sum factorisation (Section III C, Eqs. disp_expansion,
// gu_expansion, total_sf_taylor, U_fft, A_fft).
//
// For one k of the supercell grid and one site, the Taylor part of F at the voxels G = H + k of
// every zone H is the polynomial
//     S(g) = sum_{a+b+c <= P} M'_abc(k) x1^a x2^b x3^c,   x_j = g_j / gs_j,  g = H + k/n (r.l.u.),
// because the monomials are built from the displacement projected on the reciprocal axes,
// u~_j = b*_j . u, so that Q.u = g1 u~1 + g2 u~2 + g3 u~3 (the paper's own notation of Eq. gdotu_1,
// with G in r.l.u. and u in cell coordinates).  Over a box of zones this polynomial separates
// along the three grid axes and is evaluated in three contractions, each a Horner recurrence:
//     X[a,b](h3)     = sum_c M'_abc x3(h3)^c                  (P+1)(P+2)(P+3)/6 terms per h3
//     Y[a](h2,h3)    = sum_b X[a,b](h3) x2(h2)^b              (P+1)(P+2)/2 terms per (h2, h3)
//     S(h1,h2,h3)    = sum_a Y[a](h2,h3) x1(h1)^a             P+1 terms per zone
// instead of one term per monomial and zone: the same sum as Eq. total_sf_taylor, reordered
// (identical up to rounding), with about T / (P+1) times fewer multiply-adds at large order.
//
// Friedel pairs.  Only the stored half of the spectrum (k3 <= n3/2) is visited.  For a voxel whose
// k is in the other half, F(G) = conj(F(-G)) (real scattering density; it holds term by term for
// the truncated series too) and -G has a stored k: each CTA therefore evaluates its k on the zones
// of the grid (direct voxels) and on the zones of the negated grid (Friedel mates, written as
// the voxel -G with conj(F)).  When both boxes coincide (a grid symmetric about 0) one evaluation
// serves both.
//
// CTA: one stored k and one box (blockIdx.y = 0 direct, 1 mirror), 128, 256 or 512 threads, as
// many as keep 16 warps on an SM with the CTAs its shared memory admits.  Per site: the
// (a, b) chains of step 1 are spread over the threads in a balanced slot order (host table) and
// read M'(k) straight from the spectra; X and Y live in shared memory; step 3 threads own one
// (h2, h3) column each and add phi_mu(G) S into F (shared memory).  Exponents a are processed in
// groups from the highest down so that the Horner recurrence of step 3 continues across groups
// (partial S kept in shared memory when there is more than one group).  Epilogue: Bragg term at
// k = 0 (DIFFUSE), I = |F|^2 / N, one store per voxel, each voxel written by exactly one thread.
#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.h"

namespace ds {

namespace {

constexpr size_t SF_SMEM_MAX = 227 * 1024;

__device__ __forceinline__ int fdiv_floor(int a, int b) {
    int q = a / b;
    if ((a % b != 0) && ((a < 0) != (b < 0))) --q;
    return q;
}
__device__ __forceinline__ int fdiv_ceil(int a, int b) { return -fdiv_floor(-a, b); }

// acc * x + m for a complex acc and m and a real x (one paired FMA in FP32)
__device__ __forceinline__ float2 hfma(float2 acc, float x, float2 m) { return __ffma2_rn(acc, make_float2(x, x), m); }
__device__ __forceinline__ double2 hfma(double2 acc, double x, double2 m) {
    return make_double2(fma(acc.x, x, m.x), fma(acc.y, x, m.y));
}

// host: floor / ceil division
inline int hfloor(int a, int b) {
    int q = a / b;
    if ((a % b != 0) && ((a < 0) != (b < 0))) --q;
    return q;
}
inline int hceil(int a, int b) { return -hfloor(-a, b); }

// the direct and mirror zone boxes of stored k along one axis
__host__ __device__ __forceinline__ void axis_boxes(int g0, int cnt, int n, int k, int &dlo, int &dn, int &mlo,
                                                    int &mn) {
#ifdef __CUDA_ARCH__
    dlo = fdiv_ceil(g0 - k, n);
    const int dhi = fdiv_floor(g0 + cnt - 1 - k, n);
    mlo = fdiv_ceil(-(g0 + cnt - 1) - k, n);
    const int mhi = fdiv_floor(-g0 - k, n);
#else
    dlo = hceil(g0 - k, n);
    const int dhi = hfloor(g0 + cnt - 1 - k, n);
    mlo = hceil(-(g0 + cnt - 1) - k, n);
    const int mhi = hfloor(-g0 - k, n);
#endif
    dn = dhi >= dlo ? dhi - dlo + 1 : 0;
    mn = mhi >= mlo ? mhi - mlo + 1 : 0;
}

// index of the first monomial (a, b, 0) in the lexicographic list of order P
int t_index(int P, int a, int b) {
    int t = 0;
    for (int aa = 0; aa < a; ++aa) t += (P - aa + 1) * (P - aa + 2) / 2;
    for (int bb = 0; bb < b; ++bb) t += P - a - bb + 1;
    return t;
}

}  // namespace

// zone offsets of the X rows: xi(a, b) = sum_{a' = a0}^{a - 1} (P - a' + 1) + b
__host__ __device__ __forceinline__ int sf_xi(int P, int a0, int a, int b) {
    return (a - a0) * (P + 1) - (a * (a - 1) - a0 * (a0 - 1)) / 2 + b;
}

// shared-memory layout of one CTA (byte offsets, 16-byte aligned): F, S (several groups only), X,
// Y, site phases PH[site][axis][zone], Cartesian q vectors qv[axis][zone][3], x values xs[axis][zone]
struct SFLayout {
    size_t F, S, X, Y, PH, QV, XS, total;
};
__host__ __device__ __forceinline__ SFLayout sf_layout(int zr, int nsite, int xpad, int ymax, int ng, size_t ce) {
    auto al = [](size_t x) { return (x + 15) & ~(size_t)15; };
    const size_t z3 = (size_t)zr * zr * zr, re = ce / 2;
    SFLayout L;
    L.F = 0;
    L.S = al(L.F + z3 * ce);
    L.X = al(L.S + (ng > 1 ? z3 * ce : 0));
    L.Y = al(L.X + (size_t)zr * xpad * ce);
    L.PH = al(L.Y + (size_t)ymax * zr * zr * ce);
    L.QV = al(L.PH + (size_t)nsite * 3 * zr * ce);
    L.XS = al(L.QV + (size_t)9 * zr * re);
    L.total = al(L.XS + (size_t)3 * zr * re);
    return L;
}

// One CTA: stored k = blockIdx.x, box blockIdx.y (0 direct, 1 mirror).  ZR: zones per axis held in
// registers by the Horner recurrences (>= the box extents).
template <typename T, int ZR, int NT>
__global__ void __launch_bounds__(NT, 512 / NT) k_taylor_sf(const __grid_constant__ RecombParams<T> p) {
    using C = c_t<T>;
    extern __shared__ __align__(16) unsigned char smem[];
    const SFPlan &pl = p.sf;
    const Geometry &g = p.g;
    const GridMap &gm = p.gm;
    const int n1 = g.n[0], n2 = g.n[1], n3 = g.n[2], n3h = g.n3h;
    const int kidx = blockIdx.x;
    const int k1 = kidx / (n2 * n3h), krem = kidx - k1 * n2 * n3h;
    const int k2 = krem / n3h, k3 = krem - k2 * n3h;
    const int kk[3] = {k1, k2, k3};
    const int nn[3] = {n1, n2, n3};

    // boxes: direct zones of this k, and zones of the Friedel mates -G of the voxels whose k lies in
    // the unstored half (k3 in [1, n3 - n3h])
    int dlo[3], dn[3], mlo[3], mn[3];
    bool dempty = false, mempty = !(k3 >= 1 && k3 <= n3 - n3h), same = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        axis_boxes(gm.g0[a], gm.cnt[a], nn[a], kk[a], dlo[a], dn[a], mlo[a], mn[a]);
        dempty |= dn[a] == 0;
        mempty |= mn[a] == 0;
        same &= dlo[a] == mlo[a] && dn[a] == mn[a];
    }
    same &= !dempty && !mempty;
    int lo[3], nz[3];
    bool wd, wm;
    if (blockIdx.y == 0) {
        if (dempty) return;
#pragma unroll
        for (int a = 0; a < 3; ++a) lo[a] = dlo[a], nz[a] = dn[a];
        wd = true;
        wm = same;
    } else {
        if (mempty || same) return;
#pragma unroll
        for (int a = 0; a < 3; ++a) lo[a] = mlo[a], nz[a] = mn[a];
        wd = false;
        wm = true;
    }
    const int nz1 = nz[0], nz2 = nz[1], nz3 = nz[2];
    const int ncol = nz2 * nz3, nzone = nz1 * ncol;
    const int nsite = p.nsite, P = p.nT > 0 ? pl.a0[pl.ngroups] - 1 : 0;
    const SFLayout L = sf_layout(ZR, nsite, pl.xpad, pl.ymax, pl.ngroups, sizeof(C));
    C *Fs = (C *)(smem + L.F);
    C *Ss = (C *)(smem + L.S);
    C *Xs = (C *)(smem + L.X);
    C *Ys = (C *)(smem + L.Y);
    C *PH = (C *)(smem + L.PH);
    T *qv = (T *)(smem + L.QV);
    T *xs = (T *)(smem + L.XS);
    const int tid = threadIdx.x;

    // x_a(j) = (lo_a + j + k_a / n_a) / gs_a and the Cartesian q_a(j) = g_a(j) b*_a (0 beyond the box)
    for (int i = tid; i < 3 * ZR; i += NT) {
        const int a = i / ZR, j = i - a * ZR;
        const double gv = (double)(lo[a] + j) + (double)kk[a] / nn[a];
        const bool in = j < nz[a];
        xs[i] = in ? (T)(gv / p.gscale[a]) : T(0);
#pragma unroll
        for (int c = 0; c < 3; ++c) qv[3 * i + c] = in ? (T)(gv * p.recip[3 * a + c]) : T(0);
    }
    // site phases exp(2 pi i H_a r_a) per axis and zone of the box; axis 0 carries b_mu exp(ik.r_mu)
    for (int i = tid; i < nsite * 3 * ZR; i += NT) {
        const int s = i / (3 * ZR), r = i - s * 3 * ZR, a = r / ZR, j = r - a * ZR;
        const int site = p.site_of[s];
        C v = mk<T>(T(0), T(0));
        if (j < nz[a]) {
            v = p.phHx[((size_t)site * 3 + a) * p.nHx + (lo[a] + j - p.Hminx[a])];
            if (a == 0) {
                const C *tk = p.phk + (size_t)site * 3 * p.nmax;
                v = cscale(cmul(v, cmul(cmul(tk[k1], tk[p.nmax + k2]), tk[2 * p.nmax + k3])), p.scat[site]);
            }
        }
        PH[i] = v;
    }
    for (int i = tid; i < nzone; i += NT) Fs[i] = mk<T>(T(0), T(0));
    __syncthreads();

    const size_t nh = g.ncell_h;
    const bool one_ff = p.ff.ncls == 1;
    int cls = 0;
    for (int s = 0; s < nsite; ++s) {
        if (s == p.ff.cls_end[cls]) ++cls;
        const int site = p.site_of[s];
        const C *spec_s = p.spec + ((size_t)(p.model * nsite + site) * p.nT) * nh + kidx;
        for (int gi = pl.ngroups - 1; gi >= 0; --gi) {
            const int a0 = pl.a0[gi], a1 = pl.a0[gi + 1];
            // step 1: X[xi(a, b)][h3] = sum_c M'_abc x3^c, one (a, b) chain per slot
            for (int slot = pl.ibeg[gi] + tid; slot < pl.ibeg[gi + 1]; slot += NT) {
                const int4 it = pl.items[slot];
                if (it.x < 0) continue;
                const int Lc = P - it.x - it.y + 1;
                T x3[ZR];
#pragma unroll
                for (int j = 0; j < ZR; ++j) x3[j] = xs[2 * ZR + j];
                const C *src = spec_s + (size_t)it.z * nh;
                C acc[ZR];
                const C top = src[(size_t)(Lc - 1) * nh];
#pragma unroll
                for (int j = 0; j < ZR; ++j) acc[j] = top;
                constexpr int NB = sizeof(T) == 4 ? 8 : 2;  // loads in flight per thread (registers)
                for (int c = Lc - 2; c >= 0; c -= NB) {
                    C mb[NB];
#pragma unroll
                    for (int q = 0; q < NB; ++q)
                        if (c - q >= 0) mb[q] = src[(size_t)(c - q) * nh];
#pragma unroll
                    for (int q = 0; q < NB; ++q)
                        if (c - q >= 0) {
#pragma unroll
                            for (int j = 0; j < ZR; ++j) acc[j] = hfma(acc[j], x3[j], mb[q]);
                        }
                }
#pragma unroll
                for (int j = 0; j < ZR; ++j)
                    Xs[it.w * ZR + j] = acc[j];   // [item][h3], rows of ZR (odd): distinct banks
            }
            __syncthreads();
            // step 2: Y[al][h2][h3] = sum_b X[h3][xi(a, b)] x2^b, one (a, h3) per item
            const int n2it = (a1 - a0) * nz3;
            for (int i = tid; i < n2it; i += NT) {
                const int al = i / nz3, h3 = i - al * nz3;
                const int a = a0 + al, Lb = P - a + 1;
                T x2[ZR];
#pragma unroll
                for (int j = 0; j < ZR; ++j) x2[j] = xs[ZR + j];
                const C *xr = Xs + (size_t)sf_xi(P, a0, a, 0) * ZR + h3;
                C acc[ZR];
                const C top = xr[(Lb - 1) * ZR];
#pragma unroll
                for (int j = 0; j < ZR; ++j) acc[j] = top;
                for (int b = Lb - 2; b >= 0; --b) {
                    const C v = xr[b * ZR];
#pragma unroll
                    for (int j = 0; j < ZR; ++j) acc[j] = hfma(acc[j], x2[j], v);
                }
#pragma unroll
                for (int j = 0; j < ZR; ++j)
                    if (j < nz2) Ys[(al * nz2 + j) * nz3 + h3] = acc[j];
            }
            __syncthreads();
            // step 3: S(h1) = sum_a Y[a] x1^a for the thread's (h2, h3) columns, continued across groups
            for (int col = tid; col < ncol; col += NT) {
                T x1[ZR];
#pragma unroll
                for (int j = 0; j < ZR; ++j) x1[j] = xs[j];
                C Sv[ZR];
                const bool first = gi == pl.ngroups - 1;
#pragma unroll
                for (int j = 0; j < ZR; ++j) Sv[j] = (first || j >= nz1) ? mk<T>(T(0), T(0)) : Ss[j * ncol + col];
                for (int al = a1 - a0 - 1; al >= 0; --al) {
                    const C y = Ys[al * ncol + col];
#pragma unroll
                    for (int j = 0; j < ZR; ++j) Sv[j] = hfma(Sv[j], x1[j], y);
                }
                if (gi > 0) {
#pragma unroll
                    for (int j = 0; j < ZR; ++j)
                        if (j < nz1) Ss[j * ncol + col] = Sv[j];
                    continue;
                }
                // F += b f(|Q|) exp(iG.r_mu) S at the zones of this column (with one form-factor class
                // f multiplies the site sum once, in the epilogue)
                const int h2 = col / nz3, h3 = col - h2 * nz3;
                const C *ph = PH + (size_t)s * 3 * ZR;
                const C p23 = cmul(ph[ZR + h2], ph[2 * ZR + h3]);
                if (one_ff) {
#pragma unroll
                    for (int j = 0; j < ZR; ++j) {
                        if (j >= nz1) break;
                        cfma(Fs[j * ncol + col], cmul(ph[j], p23), Sv[j]);
                    }
                    continue;
                }
                T q23[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) q23[c] = qv[3 * (ZR + h2) + c] + qv[3 * (2 * ZR + h3) + c];
                const int ng = p.ff.cls_ng[cls];
#pragma unroll
                for (int j = 0; j < ZR; ++j) {
                    if (j >= nz1) break;
                    const T Qx = qv[3 * j] + q23[0], Qy = qv[3 * j + 1] + q23[1], Qz = qv[3 * j + 2] + q23[2];
                    const T q2 = Qx * Qx + Qy * Qy + Qz * Qz;
                    T f = p.ff.cls_gc[cls];
                    for (int i = 0; i < ng; ++i) f += p.ff.cls_ga[cls][i] * exp2_w(p.ff.cls_gb[cls][i] * q2);
                    const C phi = cscale(cmul(ph[j], p23), f);
                    C &Fz = Fs[j * ncol + col];
                    cfma(Fz, phi, Sv[j]);
                }
            }
        }
    }
    __syncthreads();

    // epilogue: Bragg term (DIFFUSE, k = 0), I = |F|^2 / N, direct voxel and Friedel mate
    const bool k0 = k1 == 0 && k2 == 0 && k3 == 0;
    const int g01 = gm.g0[0], g02 = gm.g0[1], g03 = gm.g0[2];
    const int c1 = gm.cnt[0], c2 = gm.cnt[1], c3 = gm.cnt[2];
    const size_t nv = (size_t)c1 * c2 * c3;
    for (int z = tid; z < nzone; z += NT) {
        const int j = z / ncol, col = z - j * ncol, h2 = col / nz3, h3 = col - h2 * nz3;
        C Fv = Fs[z];
        if (one_ff) {
            // the common form factor f(|Q|) of the zone
            T Q[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) Q[c] = qv[3 * j + c] + qv[3 * (ZR + h2) + c] + qv[3 * (2 * ZR + h3) + c];
            const T q2 = Q[0] * Q[0] + Q[1] * Q[1] + Q[2] * Q[2];
            T f = p.ff.cls_gc[0];
            for (int i = 0; i < p.ff.cls_ng[0]; ++i) f += p.ff.cls_ga[0][i] * exp2_w(p.ff.cls_gb[0][i] * q2);
            Fv = cscale(Fv, f);
        }
        const int H1 = lo[0] + j, H2 = lo[1] + h2, H3 = lo[2] + h3;
        const int G1 = n1 * H1 + k1, G2 = n2 * H2 + k2, G3 = n3 * H3 + k3;
        if (wd && G1 >= g01 && G1 < g01 + c1 && G2 >= g02 && G2 < g02 + c2 && G3 >= g03 && G3 < g03 + c3) {
            C Fd = Fv;
            if (p.diffuse && k0)
                Fd = csub(Fd, p.bragg[((size_t)(H1 - gm.Hmin[0]) * gm.nH[1] + (H2 - gm.Hmin[1])) * gm.nH[2] +
                                      (H3 - gm.Hmin[2])]);
            const size_t v = ((size_t)(G1 - g01) * c2 + (G2 - g02)) * c3 + (G3 - g03);
            const T val = p.norm * (Fd.x * Fd.x + Fd.y * Fd.y);
            p.out[v] = p.accumulate ? p.out[v] + val : val;
            if (p.Fout) p.Fout[(size_t)p.model * nv + v] = Fd;
        }
        const int M1 = -G1, M2 = -G2, M3 = -G3;
        if (wm && M1 >= g01 && M1 < g01 + c1 && M2 >= g02 && M2 < g02 + c2 && M3 >= g03 && M3 < g03 + c3) {
            const size_t v = ((size_t)(M1 - g01) * c2 + (M2 - g02)) * c3 + (M3 - g03);
            const T val = p.norm * (Fv.x * Fv.x + Fv.y * Fv.y);
            p.out[v] = p.accumulate ? p.out[v] + val : val;
            if (p.Fout) p.Fout[(size_t)p.model * nv + v] = cconj(Fv);
        }
    }
}

template <typename T, int ZR, int NT> static void launch_sf_nt(const RecombParams<T> &p, cudaStream_t s) {
    const SFLayout L = sf_layout(ZR, p.nsite, p.sf.xpad, p.sf.ymax, p.sf.ngroups, sizeof(c_t<T>));
    cudaFuncSetAttribute(k_taylor_sf<T, ZR, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.total);
    dim3 grid((unsigned)p.g.ncell_h, 2);
    k_taylor_sf<T, ZR, NT><<<grid, NT, L.total, s>>>(p);
    count_launches(1);
}

template <typename T, int ZR> static void launch_sf(const RecombParams<T> &p, cudaStream_t s) {
    if (p.sf.nthr == 128) launch_sf_nt<T, ZR, 128>(p, s);
    else if (p.sf.nthr == 256) launch_sf_nt<T, ZR, 256>(p, s);
    else launch_sf_nt<T, ZR, 512>(p, s);
}

// threads per CTA for a dynamic shared-memory footprint: 16 warps on an SM over the CTAs that fit
// (228 KB of shared memory per SM, 1 KB of it reserved per CTA)
int sf_threads_for(size_t smem) {
    const size_t fit = (228u * 1024u) / (smem + 1024u);
    return fit >= 4 ? 128 : (fit >= 2 ? 256 : 512);
}

template <typename T> void recombine_disp_sf(const RecombParams<T> &p, cudaStream_t s) {
    switch (p.sf.zr) {
        case 5: launch_sf<T, 5>(p, s); break;
        case 9: launch_sf<T, 9>(p, s); break;
        case 13: launch_sf<T, 13>(p, s); break;
        default: launch_sf<T, 17>(p, s); break;
    }
}

template void recombine_disp_sf<float>(const RecombParams<float> &, cudaStream_t);
template void recombine_disp_sf<double>(const RecombParams<double> &, cudaStream_t);

bool taylor_sf_plan(const Geometry &g, const GridMap &gm, int P, int nsite, size_t ce, bool force, SFPlan &pl,
                    std::vector<int4> &items) {
    // widest box over the stored k (direct and mirror boxes are evaluated separately unless equal)
    std::vector<int> bd[3], bm[3], bdl[3], bml[3];
    int nzmax = 0;
    for (int a = 0; a < 3; ++a) {
        const int kmax = a == 2 ? g.n3h : g.n[a];
        for (int k = 0; k < kmax; ++k) {
            int dlo, dn, mlo, mn;
            axis_boxes(gm.g0[a], gm.cnt[a], g.n[a], k, dlo, dn, mlo, mn);
            bd[a].push_back(dn);
            bm[a].push_back(mn);
            bdl[a].push_back(dlo);
            bml[a].push_back(mlo);
            nzmax = std::max(nzmax, std::max(dn, mn));
        }
    }
    const int zrs[4] = {5, 9, 13, 17};
    int zr = 0;
    for (int z : zrs)
        if (nzmax <= z) {
            zr = z;
            break;
        }
    if (!zr || P < 0) return false;
    // cost model (complex multiply-adds, the register width zr included) against the per-voxel
    // recombination, whose warps each take one k and 32 * (4 FP32, 2 FP64) of its voxels at a time
    // (T multiply-adds per voxel slot, used or not); the per-voxel kernel runs about twice as many
    // multiply-adds per second as this one (GB300), so this kernel is taken when it needs less than
    // half as many
    const double T = (double)(P + 1) * (P + 2) * (P + 3) / 6, npair = (double)(P + 1) * (P + 2) / 2;
    auto box_work = [&](int n1, int n2, int n3) {
        if (n1 == 0 || n2 == 0 || n3 == 0) return 0.0;
        return T * zr + npair * n3 * zr + (double)n2 * n3 * (P + 1) * zr;
    };
    double work_sf = 0.0;
    for (int k1 = 0; k1 < g.n[0]; ++k1)
        for (int k2 = 0; k2 < g.n[1]; ++k2)
            for (int k3 = 0; k3 < g.n3h; ++k3) {
                const bool has_m = k3 >= 1 && k3 <= g.n[2] - g.n3h;
                const bool same = has_m && bd[0][k1] == bm[0][k1] && bd[1][k2] == bm[1][k2] &&
                                  bd[2][k3] == bm[2][k3] && bdl[0][k1] == bml[0][k1] && bdl[1][k2] == bml[1][k2] &&
                                  bdl[2][k3] == bml[2][k3];
                work_sf += box_work(bd[0][k1], bd[1][k2], bd[2][k3]);
                if (has_m && !same) work_sf += box_work(bm[0][k1], bm[1][k2], bm[2][k3]);
            }
    const int slots = 32 * (ce == 16 ? 2 : 4);
    std::vector<int> vz[3];
    for (int a = 0; a < 3; ++a)
        for (int k = 0; k < g.n[a]; ++k) {
            int lo, nv, mlo, mn;
            axis_boxes(gm.g0[a], gm.cnt[a], g.n[a], k, lo, nv, mlo, mn);
            vz[a].push_back(nv);
        }
    double work_vox = 0.0;
    for (int k1 = 0; k1 < g.n[0]; ++k1)
        for (int k2 = 0; k2 < g.n[1]; ++k2) {
            const int n12 = vz[0][k1] * vz[1][k2];
            for (int k3 = 0; k3 < g.n[2]; ++k3) {
                const int nzk = n12 * vz[2][k3];
                work_vox += (double)((nzk + slots - 1) / slots) * slots;
            }
        }
    work_vox *= T;
    if (!force && 2.0 * work_sf > work_vox) return false;
    pl.zr = zr;
    const int nab = (P + 1) * (P + 2) / 2;
    auto total = [&](int nx, int na, int ng) { return sf_layout(zr, nsite, nx | 1, na, ng, ce).total; };
    // one group when everything fits, else groups (the partial S then kept in shared memory) with
    // the largest X and Y of any group within the budget
    std::vector<int> cuts;
    if (total(nab, P + 1, 1) <= SF_SMEM_MAX) {
        cuts = {0, P + 1};
    } else {
        cuts.push_back(0);
        int a = 0, xm = 0, ym = 0;
        while (a <= P) {
            int a1 = a, nit = 0;
            while (a1 <= P && total(std::max(xm, nit + (P - a1 + 1)), std::max(ym, a1 - a + 1), 2) <= SF_SMEM_MAX) {
                nit += P - a1 + 1;
                ++a1;
            }
            if (a1 == a) return false;
            xm = std::max(xm, nit);
            ym = std::max(ym, a1 - a);
            cuts.push_back(a1);
            a = a1;
        }
    }
    const int ng = (int)cuts.size() - 1;
    if (ng > SF_MAX_GROUPS) return false;
    pl.ngroups = ng;
    // footprint of the groups, then the thread count it admits
    int xmax = 0, ymax = 0;
    for (int gi = 0; gi < ng; ++gi) {
        int nc = 0;
        for (int a = cuts[gi]; a < cuts[gi + 1]; ++a) nc += P - a + 1;
        xmax = std::max(xmax, nc);
        ymax = std::max(ymax, cuts[gi + 1] - cuts[gi]);
    }
    pl.xpad = xmax | 1;
    pl.ymax = ymax;
    pl.smem = sf_layout(zr, nsite, pl.xpad, ymax, ng, ce).total;
    pl.nthr = sf_threads_for(pl.smem);
    const int NT = pl.nthr;
    items.clear();
    for (int gi = 0; gi < ng; ++gi) {
        const int a0 = cuts[gi], a1 = cuts[gi + 1];
        pl.a0[gi] = a0;
        pl.ibeg[gi] = (int)items.size();
        // chains of the group, longest first, dealt to the threads in a snake order so that every
        // thread's total chain length is about the same
        std::vector<int4> chain;
        for (int a = a0; a < a1; ++a)
            for (int b = 0; b <= P - a; ++b) chain.push_back(make_int4(a, b, t_index(P, a, b), sf_xi(P, a0, a, b)));
        std::stable_sort(chain.begin(), chain.end(),
                         [&](const int4 &u, const int4 &v) { return P - u.x - u.y > P - v.x - v.y; });
        const int nc = (int)chain.size();
        const int rounds = (nc + NT - 1) / NT;
        for (int r = 0; r < rounds; ++r)
            for (int t = 0; t < NT; ++t) {
                const int si = (r & 1) ? r * NT + (NT - 1 - t) : r * NT + t;
                items.push_back(si < nc ? chain[si] : make_int4(-1, 0, 0, 0));
            }
    }
    pl.a0[ng] = P + 1;
    pl.ibeg[ng] = (int)items.size();
    pl.items = nullptr;
    return pl.smem <= SF_SMEM_MAX;
}

}  // namespace ds
