// Residue-class recombination for sites on special positions (compositional and magnetic;
// Section III B, Eq. comp_sf_diffuse, and Section III D, Eqs. mag_sf, mag_intensity,
// mag_projection).
//
// With G = H + k (Eq. g_vec) the phase of site mu factors as exp(iH.r_mu) exp(ik.r_mu).  When
// every site's coordinate along axis a is a multiple of 1/d_a, exp(2 pi i H_a r_mu,a) depends on
// H_a only through H_a mod d_a.  For a fixed k the structure factor
//     F_c(H + k) = sum_mu exp(iH.r_mu) b_mu exp(ik.r_mu) X_mu,c(k)        (per form-factor class)
// then takes only d1 d2 d3 distinct values over all zones H: the site sum is formed once per
// residue class and every voxel of the class only adds its Q-dependent part (form factor,
// perpendicular projection, |F|^2).  This is the same sum as the per-voxel recombination, with
// the zone phases read at the class representative (the first zone of the class); the result is
// identical up to rounding.  The library picks this kernel when the classes are at least twice
// fewer than the zones; an axis without such a period counts each zone as its own class.
//
// Work split: a thread owns one k; a CTA owns 128 consecutive k, one class (rho1, rho2) of zone
// columns and a share of the rho3 classes, formed a few at a time in one pass over the sites
// (the per-site transforms are streamed from the L2-resident spectra, not kept in registers).
// Every voxel is written by exactly one thread.
#include <algorithm>

#include "internal.h"

namespace ds {

namespace {

__device__ __forceinline__ int floor_div_r(int a, int b) {
    int q = a / b;
    if ((a % b != 0) && ((a < 0) != (b < 0))) --q;
    return q;
}

constexpr int RES_THREADS = 128;
constexpr int V3 = 4;  // voxels of a residue class along axis 3 handled without a loop

// form factor of class c at |Q|^2 (Gaussian-sum form, coefficients read from the launch params);
// NG >= 0: the number of Gaussians known at compile time, NG < 0: read from the params
template <typename T, int NG>
__device__ __forceinline__ T ff_q2(const FormFactors<T> &ff, int c, T q2) {
    T f = ff.cls_gc[c];
#pragma unroll
    for (int i = 0; i < 4; ++i)
        if (NG >= 0 ? i < NG : i < ff.cls_ng[c]) f = fma(ff.cls_ga[c][i], exp2_w(ff.cls_gb[c][i] * q2), f);
    return f;
}

}  // namespace

// form factor from register-held coefficients of one class (NG Gaussians)
template <typename T, int NG>
__device__ __forceinline__ T ff_regs(const T (&ga)[4], const T (&gb)[4], T gc, T q2) {
    T f = gc;
#pragma unroll
    for (int i = 0; i < NG; ++i) f = fma(ga[i], exp2_w(gb[i] * q2), f);
    return f;
}

// MAXC: form-factor classes handled (1: one class, its form factor applied to |F|^2); D3: rho3
// classes formed per pass over the sites (their F stay in registers; Y is streamed, not kept);
// ACC: add into the output (second and later supercells of the ensemble); NG: Gaussians of the
// single form-factor class (MAXC = 1; 0 = constant form factor), -1 = read from the params.
// Launch parameters used in the voxel loops are copied to registers first.
template <typename T, int NC, int MAXC, int D3, int MINB, bool ACC, int NG>
__global__ void __launch_bounds__(RES_THREADS, MINB)
    k_recomb_cm_res(const __grid_constant__ RecombParams<T> p, int s3) {
    using C = c_t<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nsite = p.nsite;
    const int n1 = p.g.n[0], n2 = p.g.n[1], n3 = p.g.n[2];
    const int d1 = p.dres[0], d2 = p.dres[1], d3 = p.dres[2];
    const int part = blockIdx.y % s3;
    const int r12 = blockIdx.y / s3;
    const int rho1 = r12 / d2, rho2 = r12 - rho1 * d2;
    C *P123 = (C *)smem_raw;  // [d3][nsite]: exp(iH.r_mu) at the class representatives (rho1, rho2, rho3)

    for (int idx = threadIdx.x; idx < d3 * nsite; idx += blockDim.x) {
        const int r3 = idx / nsite, s = idx - r3 * nsite;
        const C *t = p.phH + (size_t)p.site_of[s] * 3 * p.nHmax;
        P123[idx] = cmul(cmul(t[rho1], t[p.nHmax + rho2]), t[2 * p.nHmax + r3]);
    }
    __syncthreads();

    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= p.g.ncell) return;
    const int k3 = k % n3;
    const int k2 = (k / n3) % n2;
    const int k1 = k / (n3 * n2);
    const int g01 = p.gm.g0[0], g02 = p.gm.g0[1], g03 = p.gm.g0[2];
    const int cnt1 = p.gm.cnt[0], cnt2 = p.gm.cnt[1], cnt3 = p.gm.cnt[2];
    const int nH1 = p.gm.nH[0], nH2 = p.gm.nH[1];
    // first voxel index along each axis of zone h: G = n (Hmin + h) + k
    const int G1b = n1 * p.gm.Hmin[0] + k1, G2b = n2 * p.gm.Hmin[1] + k2, G3b = n3 * p.gm.Hmin[2] + k3;
    // zones along axis 3 whose voxel (H3, k3) lies in the grid
    const int h3lo = max(-floor_div_r(-(g03 - G3b), n3), 0);
    const int h3hi = min(floor_div_r(g03 + cnt3 - 1 - G3b, n3), p.gm.nH[2] - 1);
    int conj;
    const int kidx = half_index(p.g, k1, k2, k3, conj);
    T qs[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) qs[i] = p.qstep[i];
    T *const out = p.out;
    const T norm = p.norm;
    T fga[4], fgb[4], fgc = T(1);
    if (MAXC == 1 && NG > 0) {
        fgc = p.ff.cls_gc[0];
#pragma unroll
        for (int i = 0; i < 4; ++i) fga[i] = p.ff.cls_ga[0][i], fgb[i] = p.ff.cls_gb[0][i];
    }
    const T dG3 = (T)(n3 * d3);  // G3 step between voxels of one residue class
    T D[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) D[a] = qs[6 + a] * dG3;
    const int stride = n3 * d3;
    const int nchunk = (d3 + D3 - 1) / D3;
    const int h3lo_mod = h3lo % d3;
    const int *const site_of = p.site_of;
    const C *const phk = p.phk;
    const T *const scat = p.scat;
    const int nmax = p.nmax, ncell_h = p.g.ncell_h;
    const C *const spec = p.spec + (size_t)p.model * nsite * NC * ncell_h + kidx;

    for (int ch = part; ch < nchunk; ch += s3) {
        const int r0 = ch * D3;
        // F of the classes rho3 = r0 .. r0 + D3 - 1, per form-factor class, one pass over the sites
        C F[D3][MAXC][NC];
#pragma unroll
        for (int r = 0; r < D3; ++r)
#pragma unroll
            for (int cl = 0; cl < MAXC; ++cl)
#pragma unroll
                for (int c = 0; c < NC; ++c) F[r][cl][c] = mk<T>(T(0), T(0));
        int cls = 0;
#pragma unroll 2
        for (int s = 0; s < nsite; ++s) {
            if (MAXC > 1 && s == p.ff.cls_end[cls]) ++cls;
            const int site = site_of[s];
            const C *t = phk + site * 3 * nmax;
            const C ph = cscale(cmul(cmul(t[k1], t[nmax + k2]), t[2 * nmax + k3]), scat[site]);
            C y[NC];
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                C x = spec[(size_t)(site * NC + c) * ncell_h];
                if (conj) x = cconj(x);
                y[c] = cmul(ph, x);
            }
#pragma unroll
            for (int r = 0; r < D3; ++r) {
                if (r0 + r < d3) {
                    const C ps = P123[(size_t)(r0 + r) * nsite + s];
#pragma unroll
                    for (int cl = 0; cl < MAXC; ++cl)
                        if (MAXC == 1 || cl == cls)
#pragma unroll
                            for (int c = 0; c < NC; ++c) cfma(F[r][cl][c], ps, y[c]);
                }
            }
        }
#pragma unroll
        for (int r = 0; r < D3; ++r) {
            const int rho3 = r0 + r;
            if (rho3 >= d3) break;
            int t3 = rho3 - h3lo_mod;
            if (t3 < 0) t3 += d3;
            const int h3s = h3lo + t3;  // first zone of the class >= h3lo
            if (h3s > h3hi) continue;
            const int nv3 = (h3hi - h3s) / d3 + 1;  // voxels of the class along axis 3
            // one class: |F|^2 (times the norm), and the part of Q.F that varies along axis 3,
            // are the same for every voxel of the residue class
            T tot1 = T(0), dpr = T(0), dpi = T(0);
            if (MAXC == 1) {
#pragma unroll
                for (int c = 0; c < NC; ++c) tot1 += F[r][0][c].x * F[r][0][c].x + F[r][0][c].y * F[r][0][c].y;
                tot1 *= norm;
                if (NC == 3) {
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        dpr = fma(D[c], F[r][0][c].x, dpr);
                        dpi = fma(D[c], F[r][0][c].y, dpi);
                    }
                }
            }
            const T tot23 = T(2) / T(3) * tot1;
            const int G3s = G3b + n3 * h3s;
            for (int h1 = rho1; h1 < nH1; h1 += d1) {
                const int G1 = G1b + n1 * h1;
                if (G1 < g01 || G1 >= g01 + cnt1) continue;
                for (int h2 = rho2; h2 < nH2; h2 += d2) {
                    const int G2 = G2b + n2 * h2;
                    if (G2 < g02 || G2 >= g02 + cnt2) continue;
                    // Q of the first voxel of the class in this column, and Q.F there
                    T Qs[3];
#pragma unroll
                    for (int a = 0; a < 3; ++a) Qs[a] = fma((T)G3s, qs[6 + a], fma((T)G1, qs[a], (T)G2 * qs[3 + a]));
                    T pr0 = T(0), pi0 = T(0);
                    if (MAXC == 1 && NC == 3) {
#pragma unroll
                        for (int c = 0; c < 3; ++c) {
                            pr0 = fma(Qs[c], F[r][0][c].x, pr0);
                            pi0 = fma(Qs[c], F[r][0][c].y, pi0);
                        }
                    }
                    T *const row = out + ((size_t)(G1 - g01) * cnt2 + (G2 - g02)) * cnt3 + (G3s - g03);
                    // voxel i3 of the class along axis 3: G3 = G3s + i3 n3 d3
                    auto voxel = [&](int i3) {
                        const T t = (T)i3;
                        T Qv[3];
#pragma unroll
                        for (int a = 0; a < 3; ++a) Qv[a] = fma(t, D[a], Qs[a]);
                        const T q2 = fma(Qv[0], Qv[0], fma(Qv[1], Qv[1], Qv[2] * Qv[2]));
                        T val;
                        if (MAXC == 1) {
                            val = tot1;
                            if (NC == 3) {
                                // |F_perp|^2 = |F|^2 - |Q.F|^2 / |Q|^2; (2/3)|F|^2 at Q = 0
                                const T pr = fma(t, dpr, pr0), pi = fma(t, dpi, pi0);
                                const T proj = fma(pr, pr, pi * pi) * (norm * rcp_w(q2));
                                val = q2 > T(0) ? tot1 - proj : tot23;
                            }
                            if (NG > 0) {
                                const T f = ff_regs<T, (NG > 0 ? NG : 0)>(fga, fgb, fgc, q2);
                                val *= f * f;
                            }
                        } else {
                            C Fv[NC];
#pragma unroll
                            for (int c = 0; c < NC; ++c) Fv[c] = mk<T>(T(0), T(0));
#pragma unroll
                            for (int cl = 0; cl < MAXC; ++cl) {
                                if (cl < p.ff.ncls) {
                                    const T f = ff_q2<T, -1>(p.ff, cl, q2);
#pragma unroll
                                    for (int c = 0; c < NC; ++c) {
                                        Fv[c].x = fma(f, F[r][cl][c].x, Fv[c].x);
                                        Fv[c].y = fma(f, F[r][cl][c].y, Fv[c].y);
                                    }
                                }
                            }
                            T tot = T(0);
#pragma unroll
                            for (int c = 0; c < NC; ++c) tot += Fv[c].x * Fv[c].x + Fv[c].y * Fv[c].y;
                            val = tot;
                            if (NC == 3) {
                                const T pr = Qv[0] * Fv[0].x + Qv[1] * Fv[1].x + Qv[2] * Fv[2].x;
                                const T pi = Qv[0] * Fv[0].y + Qv[1] * Fv[1].y + Qv[2] * Fv[2].y;
                                val = q2 > T(0) ? tot - div_w(pr * pr + pi * pi, q2) : T(2) / T(3) * tot;
                            }
                            val *= norm;
                        }
                        T *dst = row + i3 * stride;
                        if (ACC) *dst += val;
                        else *dst = val;
                    };
#pragma unroll
                    for (int i3 = 0; i3 < V3; ++i3)
                        if (i3 < nv3) voxel(i3);
                    for (int i3 = V3; i3 < nv3; ++i3) voxel(i3);
                }
            }
        }
    }
}

// shares of the rho3 chunks per CTA: a divisor of the chunk count, the smallest that gives
// `waves` waves of CTAs
static int res_split(int ctas_12, int nchunk, int slots, int waves) {
    for (int s = 1; s <= nchunk; ++s)
        if (nchunk % s == 0 && (long long)ctas_12 * s >= (long long)slots * waves) return s;
    return nchunk;
}

template <typename T, int NC, int MAXC, int D3, int MINB, bool ACC, int NG>
static void launch_res(const RecombParams<T> &p, cudaStream_t s) {
    using C = c_t<T>;
    const int ktiles = (p.g.ncell + RES_THREADS - 1) / RES_THREADS;
    const int d12 = p.dres[0] * p.dres[1];
    const int nchunk = (p.dres[2] + D3 - 1) / D3;
    const int s3 = res_split(ktiles * d12, nchunk, 152 * MINB, 1);
    const size_t sm = (size_t)p.dres[2] * p.nsite * sizeof(C);
    if (sm > 48 * 1024)
        cudaFuncSetAttribute(k_recomb_cm_res<T, NC, MAXC, D3, MINB, ACC, NG>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    dim3 grid(ktiles, d12 * s3);
    k_recomb_cm_res<T, NC, MAXC, D3, MINB, ACC, NG><<<grid, RES_THREADS, sm, s>>>(p, s3);
    count_launches(1);
}

template <typename T, int NC, int MAXC, int D3, int MINB, int NG>
static void launch_res_acc(const RecombParams<T> &p, cudaStream_t s) {
    if (p.accumulate) launch_res<T, NC, MAXC, D3, MINB, true, NG>(p, s);
    else launch_res<T, NC, MAXC, D3, MINB, false, NG>(p, s);
}

// one form-factor class: the number of its Gaussians as a compile-time constant
template <typename T, int NC, int D3, int MINB> static void launch_res_one(const RecombParams<T> &p, cudaStream_t s) {
    switch (p.ff.cls_kind[0] == 0 ? 0 : p.ff.cls_ng[0]) {
        case 0: launch_res_acc<T, NC, 1, D3, MINB, 0>(p, s); break;
        case 2: launch_res_acc<T, NC, 1, D3, MINB, 2>(p, s); break;
        case 3: launch_res_acc<T, NC, 1, D3, MINB, 3>(p, s); break;
        default: launch_res_acc<T, NC, 1, D3, MINB, 4>(p, s); break;
    }
}

template <typename T> bool recombine_cm_residues(const RecombParams<T> &p, cudaStream_t s) {
    if (p.dres[0] <= 0 || p.ff.ncls > 4 || p.force_plain || p.Fout) return false;
    if ((size_t)p.dres[2] * p.nsite * sizeof(c_t<T>) > 200 * 1024) return false;
    if ((long long)p.dres[0] * p.dres[1] * p.dres[2] > 65535) return false;  // grid.y bound
    constexpr bool dbl = sizeof(T) == 8;
    if (p.ncomp == 1) {
        if (p.ff.ncls == 1) launch_res_one<T, 1, 4, dbl ? 2 : 8>(p, s);
        else launch_res_acc<T, 1, 4, 2, dbl ? 2 : 6, -1>(p, s);
    } else {
        if (p.ff.ncls == 1) launch_res_one<T, 3, 4, dbl ? 2 : 4>(p, s);
        else launch_res_acc<T, 3, 4, 2, dbl ? 2 : 4, -1>(p, s);
    }
    return true;
}

template bool recombine_cm_residues<float>(const RecombParams<float> &, cudaStream_t);
template bool recombine_cm_residues<double>(const RecombParams<double> &, cudaStream_t);

}  // namespace ds
