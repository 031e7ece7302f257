// Recombination of the per-site transforms into F(G) and I(G) over every voxel of the
// requested commensurate grid (Section III, Eqs. total_sf_fin, comp_sf_diffuse,
// total_sf_taylor, bragg_sf_disp, mag_sf, mag_intensity, mag_projection), plus the small
// tables it needs (site phases, monomial power tables, site means, x_max for the Taylor order).
//
// Every voxel G = H + k (Eq. g_vec) is handled by exactly one thread, so no atomics are used
// and the result does not depend on scheduling.  Site phases factor as
// exp(iG.r_mu) = exp(iH.r_mu) exp(ik.r_mu), each a product of three per-axis tables computed
// in FP64 (exact reduction of the argument modulo 1) and stored in the working precision.
#include <algorithm>

#include "internal.h"

namespace ds {

// ------------------------------------------------------------------------------------------
// tables
// ------------------------------------------------------------------------------------------

template <typename T>
__global__ void k_site_tables(Geometry g, GridMap gm, int nsite, const double *sites, c_t<T> *phk, c_t<T> *phH,
                              int nmax, int nHmax) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    const int per_site = 3 * (nmax + nHmax);
    if (idx >= nsite * per_site) return;
    const int s = idx / per_site;
    int r = idx - s * per_site;
    if (r < 3 * nmax) {
        const int a = r / nmax, kk = r - a * nmax;
        if (kk >= g.n[a]) return;
        // k_a r_a / n_a, reduced exactly enough in FP64
        double t = (double)kk * sites[3 * s + a] / (double)g.n[a];
        t -= floor(t);
        double sn, cs;
        sincospi(2.0 * t, &sn, &cs);
        phk[((size_t)s * 3 + a) * nmax + kk] = mk<T>((T)cs, (T)sn);
    } else {
        r -= 3 * nmax;
        const int a = r / nHmax, hh = r - a * nHmax;
        if (hh >= gm.nH[a]) return;
        double t = (double)(gm.Hmin[a] + hh) * sites[3 * s + a];
        t -= floor(t);
        double sn, cs;
        sincospi(2.0 * t, &sn, &cs);
        phH[((size_t)s * 3 + a) * nHmax + hh] = mk<T>((T)cs, (T)sn);
    }
}

template <typename T>
void make_site_tables(const Geometry &g, const GridMap &gm, int nsite, const double *sites_dev, c_t<T> *phk,
                      c_t<T> *phH, int nmax, int nHmax, cudaStream_t s) {
    const int tot = nsite * 3 * (nmax + nHmax);
    k_site_tables<T><<<(tot + 255) / 256, 256, 0, s>>>(g, gm, nsite, sites_dev, phk, phH, nmax, nHmax);
    count_launches(1);
}

// pw[m][s][a][e][cell] = (gs_a u~_a)^e / e! with u~_a = b*_a . u the displacement projected on the
// reciprocal vector b*_a (so that Q.u = sum_a g_a u~_a for Q = sum_a g_a b*_a, Section III C), built by
// the recurrence p_e = p_{e-1} gs_a u~_a / e in FP64
struct PowerAxes {
    double b[9];   // rows b*_a (Cartesian, 1/A, including 2 pi)
    double gs[3];  // per-axis scales of the coefficients
};

template <typename T>
__global__ void k_powers(int nmodels, int nsite, int ncell, int P, const PowerAxes ax, const float *disp, T *pw) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t natom = (size_t)nmodels * nsite * ncell;
    if (idx >= natom * 3) return;
    const int a = (int)(idx / natom);
    const size_t atom = idx - (size_t)a * natom;        // (m, s, cell) linear
    const size_t ms = atom / ncell, cell = atom - ms * ncell;
    const double ut = ax.b[3 * a] * (double)disp[atom * 3] + ax.b[3 * a + 1] * (double)disp[atom * 3 + 1] +
                      ax.b[3 * a + 2] * (double)disp[atom * 3 + 2];
    const double u = ut * ax.gs[a];
    T *dst = pw + ((ms * 3 + a) * (size_t)(P + 1)) * ncell + cell;
    double p = 1.0;
    dst[0] = (T)1;
    for (int e = 1; e <= P; ++e) {
        p = p * u / (double)e;
        dst[(size_t)e * ncell] = (T)p;
    }
}

template <typename T>
void make_powers(const Geometry &g, int nmodels, int nsite, int P, const double recip[9], const double gscale[3],
                 const float *disp, T *pw, cudaStream_t s) {
    PowerAxes ax;
    for (int i = 0; i < 9; ++i) ax.b[i] = recip[i];
    for (int a = 0; a < 3; ++a) ax.gs[a] = gscale[a];
    const size_t n = (size_t)nmodels * nsite * g.ncell * 3;
    k_powers<T><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(nmodels, nsite, g.ncell, P, ax, disp, pw);
    count_launches(1);
}

__device__ __forceinline__ double block_sum(double v, double *red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
    return t;
}

// one block per (site, component): mean over supercells and lattice points, in FP64
__global__ void k_means_occ(int nmodels, int nsite, int ncell, const uint8_t *occ, double *mean) {
    __shared__ double red[32];
    const int s = blockIdx.x;
    double acc = 0.0;
    for (int m = 0; m < nmodels; ++m)
        for (int c = threadIdx.x; c < ncell; c += blockDim.x) acc += occ[((size_t)m * nsite + s) * ncell + c];
    const double t = block_sum(acc, red);
    if (threadIdx.x == 0) mean[s] = t / ((double)nmodels * ncell);
}

__global__ void k_means_spin(int nmodels, int nsite, int ncell, const float *spins, double *mean) {
    __shared__ double red[32];
    const int s = blockIdx.x / 3, a = blockIdx.x % 3;
    double acc = 0.0;
    for (int m = 0; m < nmodels; ++m)
        for (int c = threadIdx.x; c < ncell; c += blockDim.x)
            acc += spins[(((size_t)m * nsite + s) * ncell + c) * 3 + a];
    const double t = block_sum(acc, red);
    if (threadIdx.x == 0) mean[s * 3 + a] = t / ((double)nmodels * ncell);
}

void site_means_occ(int nmodels, int nsite, int ncell, const uint8_t *occ, double *mean, cudaStream_t s) {
    k_means_occ<<<nsite, 256, 0, s>>>(nmodels, nsite, ncell, occ, mean);
    count_launches(1);
}
void site_means_spin(int nmodels, int nsite, int ncell, const float *spins, double *mean, cudaStream_t s) {
    k_means_spin<<<nsite * 3, 256, 0, s>>>(nmodels, nsite, ncell, spins, mean);
    count_launches(1);
}

// out[c] = max_j |Q_c . u_j| for the 8 corners of the Q box (non-negative doubles order like
// their bit patterns, so an integer atomicMax is exact)
// out[8] = max_j |u_j| as well
__global__ void k_corner_xmax(int natom, const float *disp, const Corners cq, unsigned long long *out) {
    const double *corners = cq.v;
    double best[9];
#pragma unroll
    for (int c = 0; c < 9; ++c) best[c] = 0.0;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < natom; j += gridDim.x * blockDim.x) {
        const double ux = disp[3 * (size_t)j], uy = disp[3 * (size_t)j + 1], uz = disp[3 * (size_t)j + 2];
#pragma unroll
        for (int c = 0; c < 8; ++c)
            best[c] = fmax(best[c], fabs(corners[3 * c] * ux + corners[3 * c + 1] * uy + corners[3 * c + 2] * uz));
        best[8] = fmax(best[8], sqrt(ux * ux + uy * uy + uz * uz));
    }
#pragma unroll
    for (int c = 0; c < 9; ++c) {
        double v = best[c];
        for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
        if ((threadIdx.x & 31) == 0) atomicMax(out + c, (unsigned long long)__double_as_longlong(v));
    }
}

void corner_xmax(int natom, const float *disp, const Corners &corners, double *out, cudaStream_t s) {
    cudaMemsetAsync(out, 0, 9 * sizeof(double), s);
    int nb = std::min(1024, std::max(1, (natom + 255) / 256));
    k_corner_xmax<<<nb, 256, 0, s>>>(natom, disp, corners, (unsigned long long *)out);
    count_launches(1);
}

// ------------------------------------------------------------------------------------------
// helpers shared by the recombination kernels
// ------------------------------------------------------------------------------------------

__device__ __forceinline__ int floor_div(int a, int b) {
    int q = a / b;
    if ((a % b != 0) && ((a < 0) != (b < 0))) --q;
    return q;
}
__device__ __forceinline__ int ceil_div(int a, int b) { return -floor_div(-a, b); }

// Cartesian Q of G (supercell indices) in FP64
__device__ __forceinline__ void q_of_G(const double *recip, const int *n, int G1, int G2, int G3, double *Q) {
    const double h = (double)G1 / n[0], k = (double)G2 / n[1], l = (double)G3 / n[2];
#pragma unroll
    for (int a = 0; a < 3; ++a) Q[a] = h * recip[a] + k * recip[3 + a] + l * recip[6 + a];
}
// scaled Taylor coefficients' variables x_a = (G_a / n_a) / gscale_a (|x_a| <= 1 on the grid)
__device__ __forceinline__ void x_of_G(const double *gscale, const int *n, int G1, int G2, int G3, double *x) {
    x[0] = (double)G1 / n[0] / gscale[0];
    x[1] = (double)G2 / n[1] / gscale[1];
    x[2] = (double)G3 / n[2] / gscale[2];
}

// ------------------------------------------------------------------------------------------
// compositional (NC = 1) and magnetic (NC = 3) recombination
// ------------------------------------------------------------------------------------------
// CTA: 256 consecutive k (k3 fastest) x a chunk of (H1, H2) zone columns; each thread keeps
// Y_mu,c(k) = b_mu exp(ik.r_mu) X_mu,c(k) of its k in registers and sweeps the zones, reading
// exp(iH.r_mu) from a shared-memory table that every thread of the warp reads at once.

template <typename T> struct CmConfig {
    int h12_per_cta;
};

// One voxel pass of the site sum for VPI consecutive h3 zones, then the epilogue.
// ONECLS: every site shares one form factor (applied once after the site sum).
template <typename T, int NC, int MAXS, bool ONECLS, int VPI, int MINB>
__global__ void __launch_bounds__(256, MINB)
    k_recomb_cm(const __grid_constant__ RecombParams<T> p, int h12_per_cta) {
    using C = c_t<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int cls_end_s[MAX_FF_CLASSES];
    __shared__ int cls_kind_s[MAX_FF_CLASSES];
    __shared__ T cls_coef_s[MAX_FF_CLASSES][9];
    C *Ptab = (C *)smem_raw;
    const Geometry &g = p.g;
    const GridMap &gm = p.gm;
    const int nsite = p.nsite;
    const int nH12 = gm.nH[0] * gm.nH[1];
    const int h12_0 = blockIdx.y * h12_per_cta;
    const int nh12 = min(h12_per_cta, nH12 - h12_0);
    const int nH3 = gm.nH[2];

    if (threadIdx.x < MAX_FF_CLASSES) {
        cls_end_s[threadIdx.x] = p.ff.cls_end[threadIdx.x];
        cls_kind_s[threadIdx.x] = p.ff.cls_kind[threadIdx.x];
#pragma unroll
        for (int j = 0; j < 9; ++j) cls_coef_s[threadIdx.x][j] = p.ff.cls_coef[threadIdx.x][j];
    }
    for (int idx = threadIdx.x; idx < nh12 * nH3 * nsite; idx += blockDim.x) {
        const int s = idx % nsite;
        const int h3 = (idx / nsite) % nH3;
        const int j12 = idx / (nsite * nH3);
        const int h12 = h12_0 + j12;
        const int h1 = h12 / gm.nH[1], h2 = h12 - h1 * gm.nH[1];
        const int site = p.site_of[s];
        const C *t = p.phH + (size_t)site * 3 * p.nHmax;
        Ptab[idx] = cmul(cmul(t[h1], t[p.nHmax + h2]), t[2 * p.nHmax + h3]);
    }
    __syncthreads();

    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= g.ncell) return;
    const int k3 = k % g.n[2];
    const int k2 = (k / g.n[2]) % g.n[1];
    const int k1 = k / (g.n[2] * g.n[1]);

    // zones along axis 3 reachable from this k3
    int h3lo = ceil_div(gm.g0[2] - k3, g.n[2]) - gm.Hmin[2];
    int h3hi = floor_div(gm.g0[2] + gm.cnt[2] - 1 - k3, g.n[2]) - gm.Hmin[2];
    h3lo = max(h3lo, 0);
    h3hi = min(h3hi, nH3 - 1);

    int conj;
    const int kidx = half_index(g, k1, k2, k3, conj);
    C Y[MAXS][NC];
#pragma unroll
    for (int s = 0; s < MAXS; ++s) {
        if (s < nsite) {
            const int site = p.site_of[s];
            const C *t = p.phk + (size_t)site * 3 * p.nmax;
            const C ph = cscale(cmul(cmul(t[k1], t[p.nmax + k2]), t[2 * p.nmax + k3]), p.scat[site]);
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                C x = p.spec[(((size_t)p.model * nsite + site) * NC + c) * g.ncell_h + kidx];
                if (conj) x = cconj(x);
                Y[s][c] = cmul(ph, x);
            }
        } else {
#pragma unroll
            for (int c = 0; c < NC; ++c) Y[s][c] = mk<T>(T(0), T(0));
        }
    }
    const int kind0 = cls_kind_s[0];
    const T inv16pi2 = (T)(1.0 / (FOUR_PI_D * FOUR_PI_D));

    for (int j12 = 0; j12 < nh12; ++j12) {
        const int h12 = h12_0 + j12;
        const int h1 = h12 / gm.nH[1], h2 = h12 - h1 * gm.nH[1];
        const int G1 = g.n[0] * (gm.Hmin[0] + h1) + k1;
        const int G2 = g.n[1] * (gm.Hmin[1] + h2) + k2;
        if (G1 < gm.g0[0] || G1 >= gm.g0[0] + gm.cnt[0]) continue;
        if (G2 < gm.g0[1] || G2 >= gm.g0[1] + gm.cnt[1]) continue;
        const C *Prow = Ptab + (size_t)j12 * nH3 * nsite;
        const long long row0 = ((long long)(G1 - gm.g0[0]) * gm.cnt[1] + (G2 - gm.g0[1])) * gm.cnt[2] - gm.g0[2];
        T *orow = p.out + row0;
        // Debye-Waller factor T_mu(G) of this row (magnetic + displacive coupling, Eq. mag_sf)
        const T *dwrow = p.dw ? p.dw + row0 : nullptr;
        const long long dw_site_stride = (long long)gm.cnt[0] * gm.cnt[1] * gm.cnt[2];
        // Cartesian Q = (G1/n1) a* + (G2/n2) b* + (G3/n3) c*, the G3 part added per voxel
        T Q12[3], c3[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            Q12[a] = fma((T)G1, p.qstep[a], (T)G2 * p.qstep[3 + a]);
            c3[a] = p.qstep[6 + a];
        }
        for (int h3 = h3lo; h3 <= h3hi; h3 += VPI) {
            C F[VPI][NC], part[VPI][NC];
#pragma unroll
            for (int v = 0; v < VPI; ++v)
#pragma unroll
                for (int c = 0; c < NC; ++c) F[v][c] = part[v][c] = mk<T>(T(0), T(0));
            T s2[VPI], Qv[VPI][3], q2[VPI];
#pragma unroll
            for (int v = 0; v < VPI; ++v) {
                const int G3 = g.n[2] * (gm.Hmin[2] + min(h3 + v, h3hi)) + k3;
#pragma unroll
                for (int a = 0; a < 3; ++a) Qv[v][a] = fma((T)G3, c3[a], Q12[a]);
                q2[v] = Qv[v][0] * Qv[v][0] + Qv[v][1] * Qv[v][1] + Qv[v][2] * Qv[v][2];
                s2[v] = q2[v] * inv16pi2;
            }
            int cls = 0;
#pragma unroll
            for (int s = 0; s < MAXS; ++s) {
                if (s < nsite) {
#pragma unroll
                    for (int v = 0; v < VPI; ++v) {
                        C ps = Prow[(size_t)min(h3 + v, h3hi) * nsite + s];
                        if (dwrow)
                            ps = cscale(ps, dwrow[(long long)p.site_of[s] * dw_site_stride +
                                                  (long long)(g.n[2] * (gm.Hmin[2] + min(h3 + v, h3hi)) + k3)]);
                        if (ONECLS) {
#pragma unroll
                            for (int c = 0; c < NC; ++c) cfma(F[v][c], ps, Y[s][c]);
                        } else {
#pragma unroll
                            for (int c = 0; c < NC; ++c) cfma(part[v][c], ps, Y[s][c]);
                        }
                    }
                    if (!ONECLS && s + 1 == cls_end_s[cls]) {
#pragma unroll
                        for (int v = 0; v < VPI; ++v) {
                            const T f = form_factor<T>(cls_kind_s[cls], cls_coef_s[cls], s2[v]);
#pragma unroll
                            for (int c = 0; c < NC; ++c) {
                                F[v][c].x = fma(f, part[v][c].x, F[v][c].x);
                                F[v][c].y = fma(f, part[v][c].y, F[v][c].y);
                                part[v][c] = mk<T>(T(0), T(0));
                            }
                        }
                        ++cls;
                    }
                }
            }
#pragma unroll
            for (int v = 0; v < VPI; ++v) {
                if (h3 + v > h3hi) break;
                T tot = T(0);
#pragma unroll
                for (int c = 0; c < NC; ++c) tot += F[v][c].x * F[v][c].x + F[v][c].y * F[v][c].y;
                T I = tot;
                if (NC == 3) {
                    if (q2[v] > T(0)) {
                        const T pr = Qv[v][0] * F[v][0].x + Qv[v][1] * F[v][1].x + Qv[v][2] * F[v][2].x;
                        const T pi = Qv[v][0] * F[v][0].y + Qv[v][1] * F[v][1].y + Qv[v][2] * F[v][2].y;
                        I = tot - div_w(pr * pr + pi * pi, q2[v]);
                    } else {
                        I = T(2) / T(3) * tot;
                    }
                }
                T fone = T(1);
                if (ONECLS && kind0 != 0) {
                    fone = form_factor<T>(kind0, cls_coef_s[0], s2[v]);
                    I *= fone * fone;
                }
                T *dst = orow + g.n[2] * (gm.Hmin[2] + h3 + v) + k3;
                const T val = p.norm * I;
                *dst = p.accumulate ? *dst + val : val;
                if (p.Fout) {
                    const size_t vi = (size_t)(dst - p.out);
                    const size_t nv = (size_t)gm.cnt[0] * gm.cnt[1] * gm.cnt[2];
#pragma unroll
                    for (int c = 0; c < NC; ++c)
                        p.Fout[((size_t)p.model * nv + vi) * NC + c] = cscale(F[v][c], fone);
                }
            }
        }
    }
}

template <typename T, int NC, int MAXS, bool ONECLS, int VPI, int MINB>
void launch_cm_variant(const RecombParams<T> &p, int per, cudaStream_t s) {
    using C = c_t<T>;
    const int nH12 = p.gm.nH[0] * p.gm.nH[1];
    const int ktiles = (p.g.ncell + 255) / 256;
    const size_t sm = (size_t)per * p.gm.nH[2] * p.nsite * sizeof(C);
    if (sm > 48 * 1024)
        cudaFuncSetAttribute(k_recomb_cm<T, NC, MAXS, ONECLS, VPI, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sm);
    dim3 grid(ktiles, (nH12 + per - 1) / per);
    k_recomb_cm<T, NC, MAXS, ONECLS, VPI, MINB><<<grid, 256, sm, s>>>(p, per);
    count_launches(1);
}

// Grouped variant: per (k, H1, H2) column the site sum is first reduced to one partial sum per
// site group (sites of one form-factor class sharing z = r_mu,3 mod 1),
//     A_g,c = sum_{mu in g} exp(2 pi i (H1 x_mu + H2 y_mu)) Y_mu,c(k),
// and each voxel of the column then needs only
//     F_c(H + k) = sum_g exp(2 pi i H3 z_g) A_g,c
// (times the class form factor), i.e. n_groups instead of n_sites complex multiply-adds.
template <typename T, int NC, int MAXS, int MAXG, bool ONECLS, int VPI, int MINB, bool YSMEM>
__global__ void __launch_bounds__(256, MINB)
    k_recomb_cm_grp(const __grid_constant__ RecombParams<T> p, int h12_per_cta) {
    using C = c_t<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int grp_end_s[MAX_SITES];
    __shared__ int cls_grp_end_s[MAX_FF_CLASSES];
    __shared__ int cls_kind_s[MAX_FF_CLASSES];
    __shared__ T cls_coef_s[MAX_FF_CLASSES][9];
    const Geometry &g = p.g;
    const GridMap &gm = p.gm;
    const int nsite = p.nsite, ngrp = p.grp.ngrp;
    const int nH12 = gm.nH[0] * gm.nH[1];
    const int h12_0 = blockIdx.y * h12_per_cta;
    const int nh12 = min(h12_per_cta, nH12 - h12_0);
    const int nH3 = gm.nH[2];
    C *P12 = (C *)smem_raw;                           // [per][nsite]
    C *W = P12 + (size_t)h12_per_cta * nsite;         // [nH3 + 1][ngrp]
    C *Ys = W + (size_t)(nH3 + 1) * ngrp;             // YSMEM: [nsite][NC][256]

    if (threadIdx.x < MAX_SITES) grp_end_s[threadIdx.x] = p.grp.grp_end[threadIdx.x];
    if (threadIdx.x < MAX_FF_CLASSES) {
        cls_grp_end_s[threadIdx.x] = p.grp.cls_grp_end[threadIdx.x];
        cls_kind_s[threadIdx.x] = p.ff.cls_kind[threadIdx.x];
#pragma unroll
        for (int j = 0; j < 9; ++j) cls_coef_s[threadIdx.x][j] = p.ff.cls_coef[threadIdx.x][j];
    }
    for (int idx = threadIdx.x; idx < nh12 * nsite; idx += blockDim.x) {
        const int s = idx % nsite, j12 = idx / nsite;
        const int h12 = h12_0 + j12;
        const int h1 = h12 / gm.nH[1], h2 = h12 - h1 * gm.nH[1];
        const C *t = p.phH + (size_t)p.site_of[s] * 3 * p.nHmax;
        P12[idx] = cmul(t[h1], t[p.nHmax + h2]);
    }
    for (int idx = threadIdx.x; idx < (nH3 + 1) * ngrp; idx += blockDim.x) {
        const int gg = idx % ngrp, h3 = idx / ngrp;
        if (h3 < nH3) {
            W[idx] = p.phH[((size_t)p.grp.grp_site[gg] * 3 + 2) * p.nHmax + h3];
        } else {
            // exp(2 pi i z_g), z_g = r_3 mod 1 of the group's site
            double z = p.sites[3 * p.grp.grp_site[gg] + 2];
            z -= floor(z);
            double sn, cs;
            sincospi(2.0 * z, &sn, &cs);
            W[idx] = mk<T>((T)cs, (T)sn);
        }
    }
    __syncthreads();

    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= g.ncell) return;
    const int k3 = k % g.n[2];
    const int k2 = (k / g.n[2]) % g.n[1];
    const int k1 = k / (g.n[2] * g.n[1]);
    int h3lo = ceil_div(gm.g0[2] - k3, g.n[2]) - gm.Hmin[2];
    int h3hi = floor_div(gm.g0[2] + gm.cnt[2] - 1 - k3, g.n[2]) - gm.Hmin[2];
    h3lo = max(h3lo, 0);
    h3hi = min(h3hi, nH3 - 1);

    int conj;
    const int kidx = half_index(g, k1, k2, k3, conj);
    C Y[YSMEM ? 1 : MAXS][NC];
#pragma unroll
    for (int s = 0; s < MAXS; ++s) {
        if (s < nsite) {
            const int site = p.site_of[s];
            const C *t = p.phk + (size_t)site * 3 * p.nmax;
            const C ph = cscale(cmul(cmul(t[k1], t[p.nmax + k2]), t[2 * p.nmax + k3]), p.scat[site]);
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                C x = p.spec[(((size_t)p.model * nsite + site) * NC + c) * g.ncell_h + kidx];
                if (conj) x = cconj(x);
                if (YSMEM) Ys[((size_t)s * NC + c) * 256 + threadIdx.x] = cmul(ph, x);
                else Y[YSMEM ? 0 : s][c] = cmul(ph, x);
            }
        } else if (!YSMEM) {
#pragma unroll
            for (int c = 0; c < NC; ++c) Y[YSMEM ? 0 : s][c] = mk<T>(T(0), T(0));
        }
    }
    const int kind0 = cls_kind_s[0];
    const T inv16pi2 = (T)(1.0 / (FOUR_PI_D * FOUR_PI_D));

    for (int j12 = 0; j12 < nh12; ++j12) {
        const int h12 = h12_0 + j12;
        const int h1 = h12 / gm.nH[1], h2 = h12 - h1 * gm.nH[1];
        const int G1 = g.n[0] * (gm.Hmin[0] + h1) + k1;
        const int G2 = g.n[1] * (gm.Hmin[1] + h2) + k2;
        if (G1 < gm.g0[0] || G1 >= gm.g0[0] + gm.cnt[0]) continue;
        if (G2 < gm.g0[1] || G2 >= gm.g0[1] + gm.cnt[1]) continue;
        // group sums of this column
        C A[MAXG][NC];
#pragma unroll
        for (int gg = 0; gg < MAXG; ++gg)
#pragma unroll
            for (int c = 0; c < NC; ++c) A[gg][c] = mk<T>(T(0), T(0));
        {
            const C *Pr = P12 + (size_t)j12 * nsite;
            C part[NC];
#pragma unroll
            for (int c = 0; c < NC; ++c) part[c] = mk<T>(T(0), T(0));
            int gcur = 0;
#pragma unroll
            for (int s = 0; s < MAXS; ++s) {
                if (s < nsite) {
                    const C ps = Pr[s];
#pragma unroll
                    for (int c = 0; c < NC; ++c) {
                        const C y = YSMEM ? Ys[((size_t)s * NC + c) * 256 + threadIdx.x] : Y[YSMEM ? 0 : s][c];
                        cfma(part[c], ps, y);
                    }
                    if (s + 1 == grp_end_s[gcur]) {
#pragma unroll
                        for (int gg = 0; gg < MAXG; ++gg)
                            if (gg == gcur)
#pragma unroll
                                for (int c = 0; c < NC; ++c) A[gg][c] = part[c];
#pragma unroll
                        for (int c = 0; c < NC; ++c) part[c] = mk<T>(T(0), T(0));
                        ++gcur;
                    }
                }
            }
        }
        T *orow = p.out + ((size_t)(G1 - gm.g0[0]) * gm.cnt[1] + (G2 - gm.g0[1])) * gm.cnt[2] - gm.g0[2];
        T Q12[3], c3[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            Q12[a] = fma((T)G1, p.qstep[a], (T)G2 * p.qstep[3 + a]);
            c3[a] = p.qstep[6 + a];
        }
        // exp(2 pi i H3 z_g) of the first voxel, then advanced by exp(2 pi i z_g) per zone step
        C wcur[MAXG], wstep[MAXG];
#pragma unroll
        for (int gg = 0; gg < MAXG; ++gg) {
            if (gg < ngrp) {
                wcur[gg] = W[h3lo * ngrp + gg];
                wstep[gg] = W[nH3 * ngrp + gg];
            }
        }
        for (int h3 = h3lo; h3 <= h3hi; h3 += VPI) {
            C F[VPI][NC], part[VPI][NC];
            T s2[VPI], Qv[VPI][3], q2[VPI];
#pragma unroll
            for (int v = 0; v < VPI; ++v) {
                const int G3 = g.n[2] * (gm.Hmin[2] + h3 + v) + k3;
#pragma unroll
                for (int a = 0; a < 3; ++a) Qv[v][a] = fma((T)G3, c3[a], Q12[a]);
                q2[v] = Qv[v][0] * Qv[v][0] + Qv[v][1] * Qv[v][1] + Qv[v][2] * Qv[v][2];
                s2[v] = q2[v] * inv16pi2;
#pragma unroll
                for (int c = 0; c < NC; ++c) F[v][c] = part[v][c] = mk<T>(T(0), T(0));
            }
            int cls = 0;
#pragma unroll
            for (int gg = 0; gg < MAXG; ++gg) {
                if (gg < ngrp) {
#pragma unroll
                    for (int v = 0; v < VPI; ++v) {
                        const C w = wcur[gg];
#pragma unroll
                        for (int c = 0; c < NC; ++c) cfma(ONECLS ? F[v][c] : part[v][c], w, A[gg][c]);
                        wcur[gg] = cmul(wcur[gg], wstep[gg]);
                    }
                    if (!ONECLS && gg + 1 == cls_grp_end_s[cls]) {
#pragma unroll
                        for (int v = 0; v < VPI; ++v) {
                            const T f = form_factor<T>(cls_kind_s[cls], cls_coef_s[cls], s2[v]);
#pragma unroll
                            for (int c = 0; c < NC; ++c) {
                                F[v][c].x = fma(f, part[v][c].x, F[v][c].x);
                                F[v][c].y = fma(f, part[v][c].y, F[v][c].y);
                                part[v][c] = mk<T>(T(0), T(0));
                            }
                        }
                        ++cls;
                    }
                }
            }
            T val[VPI];
#pragma unroll
            for (int v = 0; v < VPI; ++v) {
                T tot = T(0);
#pragma unroll
                for (int c = 0; c < NC; ++c) tot += F[v][c].x * F[v][c].x + F[v][c].y * F[v][c].y;
                T I = tot;
                if (NC == 3) {
                    const T pr = Qv[v][0] * F[v][0].x + Qv[v][1] * F[v][1].x + Qv[v][2] * F[v][2].x;
                    const T pi = Qv[v][0] * F[v][0].y + Qv[v][1] * F[v][1].y + Qv[v][2] * F[v][2].y;
                    I = q2[v] > T(0) ? tot - div_w(pr * pr + pi * pi, q2[v]) : T(2) / T(3) * tot;
                }
                if (ONECLS && kind0 != 0) {
                    const T f = form_factor<T>(kind0, cls_coef_s[0], s2[v]);
                    I *= f * f;
                }
                val[v] = p.norm * I;
            }
#pragma unroll
            for (int v = 0; v < VPI; ++v) {
                if (h3 + v <= h3hi) {
                    T *dst = orow + g.n[2] * (gm.Hmin[2] + h3 + v) + k3;
                    *dst = p.accumulate ? *dst + val[v] : val[v];
                }
            }
        }
    }
}

template <typename T, int NC, int MAXS, int MAXG, bool ONECLS, int VPI, int MINB, bool YSMEM = false>
void launch_cm_grp_variant(const RecombParams<T> &p, int per, cudaStream_t s) {
    using C = c_t<T>;
    const int nH12 = p.gm.nH[0] * p.gm.nH[1];
    const int ktiles = (p.g.ncell + 255) / 256;
    size_t sm = ((size_t)per * p.nsite + (size_t)(p.gm.nH[2] + 1) * p.grp.ngrp) * sizeof(C);
    if (YSMEM) sm += (size_t)p.nsite * NC * 256 * sizeof(C);
    if (sm > 48 * 1024)
        cudaFuncSetAttribute(k_recomb_cm_grp<T, NC, MAXS, MAXG, ONECLS, VPI, MINB, YSMEM>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    dim3 grid(ktiles, (nH12 + per - 1) / per);
    k_recomb_cm_grp<T, NC, MAXS, MAXG, ONECLS, VPI, MINB, YSMEM><<<grid, 256, sm, s>>>(p, per);
    count_launches(1);
}

// (H1, H2) columns per CTA: enough CTAs for several waves, shared table within budget
template <typename T> static int cm_columns_per_cta(const RecombParams<T> &p, int waves_target) {
    using C = c_t<T>;
    const int nH12 = p.gm.nH[0] * p.gm.nH[1];
    const int ktiles = (p.g.ncell + 255) / 256;
    int per = std::max(1, (nH12 * ktiles) / (152 * waves_target));
    per = std::min(per, nH12);
    while ((size_t)per * p.gm.nH[2] * p.nsite * sizeof(C) > 96 * 1024 && per > 1) per = (per + 1) / 2;
    return per;
}

template <typename T, int NC, int MAXS> static void launch_cm(const RecombParams<T> &p, cudaStream_t s) {
    const int per = cm_columns_per_cta<T>(p, 8);
    const bool one = p.ff.ncls == 1;
    const int ng = p.force_plain ? p.nsite : p.grp.ngrp;
    // grouping pays when the groups are at most half the sites
    // measured on GB300 (16 sites, 20^3 cells, 241^3 voxels): magnetic fastest with 2 CTAs/SM
    // and Y in registers; occupancy with Y staged in shared memory and 4 CTAs/SM
    if (2 * ng <= p.nsite && ng <= 8) {
        const int per4 = cm_columns_per_cta<T>(p, 4);
        if (NC == 3) {
            if (ng <= 4) {
                if (one) launch_cm_grp_variant<T, NC, MAXS, 4, true, 1, 2>(p, per4, s);
                else launch_cm_grp_variant<T, NC, MAXS, 4, false, 1, 2>(p, per4, s);
            } else {
                if (one) launch_cm_grp_variant<T, NC, MAXS, 8, true, 1, 2>(p, per4, s);
                else launch_cm_grp_variant<T, NC, MAXS, 8, false, 1, 2>(p, per4, s);
            }
        } else {
            if (ng <= 4) {
                if (one) launch_cm_grp_variant<T, NC, MAXS, 4, true, 1, 4, true>(p, per4, s);
                else launch_cm_grp_variant<T, NC, MAXS, 4, false, 1, 4, true>(p, per4, s);
            } else {
                if (one) launch_cm_grp_variant<T, NC, MAXS, 8, true, 1, 4, true>(p, per4, s);
                else launch_cm_grp_variant<T, NC, MAXS, 8, false, 1, 4, true>(p, per4, s);
            }
        }
        return;
    }
    if (one) launch_cm_variant<T, NC, MAXS, true, NC == 3 ? 2 : 1, 2>(p, per, s);
    else launch_cm_variant<T, NC, MAXS, false, 1, 2>(p, per, s);
}

template <typename T> void recombine_cm(const RecombParams<T> &p, cudaStream_t s) {
    if (recombine_rows<T>(p, s)) return;
    if (recombine_cm_residues<T>(p, s)) return;
    if (p.ncomp == 1) {
        if (p.nsite <= 4) launch_cm<T, 1, 4>(p, s);
        else if (p.nsite <= 8) launch_cm<T, 1, 8>(p, s);
        else if (p.nsite <= 16) launch_cm<T, 1, 16>(p, s);
        else launch_cm<T, 1, 32>(p, s);
    } else {
        if (p.nsite <= 4) launch_cm<T, 3, 4>(p, s);
        else if (p.nsite <= 8) launch_cm<T, 3, 8>(p, s);
        else launch_cm<T, 3, 16>(p, s);
    }
}

// ------------------------------------------------------------------------------------------
// displacive (Taylor) recombination
// ------------------------------------------------------------------------------------------
// CTA: KT consecutive k (one warp each) x a chunk of 32*ZPT zones of each k's own zone box.
// The transforms M_mu,t(k) of the CTA's k are staged TC monomials at a time in shared memory
// by asynchronous copies, double buffered (the next chunk is in flight while the current one is
// used), and read by all lanes of a warp at once.  Each lane keeps the scaled coefficients
// x1^a x2^b x3^c (x_j = g_j / gs_j, g the r.l.u. coordinates of G) of its ZPT voxels, updated with
// one multiply per monomial
// (monomials run in lexicographic (a, b, c) order), and accumulates S_mu += coef * M_mu,t.
// A k of the other half of the spectrum reads the stored i^n M(-k): its value is
// (-1)^n conj(stored), applied with compile-time signs in a separate loop body.

constexpr int DISP_KT = 8;
constexpr int DISP_TC = 32;
enum { OP_MULZ = 0, OP_NEWB = 1, OP_NEWA = 2, OP_INIT = 3 };

struct ZoneBox {
    int lo[3], n[3];
};

__device__ __forceinline__ ZoneBox zone_box(const Geometry &g, const GridMap &gm, int k1, int k2, int k3) {
    ZoneBox b;
    const int kk[3] = {k1, k2, k3};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int lo = ceil_div(gm.g0[a] - kk[a], g.n[a]);
        const int hi = floor_div(gm.g0[a] + gm.cnt[a] - 1 - kk[a], g.n[a]);
        b.lo[a] = lo;
        b.n[a] = max(0, hi - lo + 1);
    }
    return b;
}

// one chunk of monomials for one warp; CONJ: the warp's k reads the mirrored half spectrum;
// MASK: a voxel takes only the monomials of order n <= its zone's order pzv[j].  The update code
// and the order of a monomial are the same for the whole warp, so each is a uniform branch and
// the per-voxel work is one coefficient multiply and 2 NS multiply-adds.
// Coefficient arithmetic of the Taylor recombination.  FP32 keeps the running coefficient of the
// current monomial as a duplicated pair (c, c), so that S += c m is one paired FMA (FFMA2) on
// the complex S and the coefficient update one paired multiply; FP64 uses scalars.
template <typename T> struct CoefPair { using type = T; };
template <> struct CoefPair<float> { using type = float2; };
__device__ __forceinline__ float2 pair_of(float v) { return make_float2(v, v); }
__device__ __forceinline__ double pair_of(double v) { return v; }
__device__ __forceinline__ float2 pair_mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ double pair_mul(double a, double b) { return a * b; }
__device__ __forceinline__ void pair_acc(float2 &S, float2 w, float2 m) { S = __ffma2_rn(w, m, S); }
__device__ __forceinline__ void pair_acc(double2 &S, double w, double2 m) {
    S.x = fma(w, m.x, S.x);
    S.y = fma(w, m.y, S.y);
}

// one chunk of monomials for one warp; MASK: a voxel takes only the monomials of order
// n <= its zone's order pzv[j].  The update code and the order of a monomial are the same for the
// whole warp (uniform branches); per voxel and monomial the work is one coefficient multiply and
// NS complex multiply-adds.
template <typename T, int NS, int ZPT, bool MASK>
__device__ __forceinline__ void disp_chunk(const c_t<T> *wt, const int *tinfo, int tc, const T (&qx)[ZPT],
                                           const T (&qy)[ZPT], const typename CoefPair<T>::type (&qzp)[ZPT],
                                           const int (&pzv)[ZPT], T (&ca)[ZPT], T (&cb)[ZPT],
                                           typename CoefPair<T>::type (&ccp)[ZPT], c_t<T> (&S)[ZPT][NS]) {
    using P = typename CoefPair<T>::type;
    for (int tt = 0; tt < tc; ++tt) {
        const int info = tinfo[tt];
        const int op = info & 3;
        const int n = info >> 2;
        if (op == OP_MULZ) {
#pragma unroll
            for (int j = 0; j < ZPT; ++j) ccp[j] = pair_mul(ccp[j], qzp[j]);
        } else if (op == OP_NEWB) {
#pragma unroll
            for (int j = 0; j < ZPT; ++j) {
                cb[j] *= qy[j];
                ccp[j] = pair_of(cb[j]);
            }
        } else if (op == OP_NEWA) {
#pragma unroll
            for (int j = 0; j < ZPT; ++j) {
                ca[j] *= qx[j];
                cb[j] = ca[j];
                ccp[j] = pair_of(ca[j]);
            }
        } else {
#pragma unroll
            for (int j = 0; j < ZPT; ++j) {
                ca[j] = cb[j] = T(1);
                ccp[j] = pair_of(T(1));
            }
        }
        P w[ZPT];
#pragma unroll
        for (int j = 0; j < ZPT; ++j) w[j] = (!MASK || n <= pzv[j]) ? ccp[j] : pair_of(T(0));
        const c_t<T> *mt = wt + tt;
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            const c_t<T> m = mt[s * DISP_TC];
#pragma unroll
            for (int j = 0; j < ZPT; ++j) pair_acc(S[j][s], w[j], m);
        }
    }
}

// NS: sites held per thread (the tile keeps NS rows; rows beyond nsite are zero); MINB: CTAs per
// SM the register budget is sized for
template <typename T, int NS, int ZPT, int MINB>
__global__ void __launch_bounds__(DISP_KT * 32, MINB) k_recomb_disp(const __grid_constant__ RecombParams<T> p) {
    using C = c_t<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int kidx_s[DISP_KT], kconj_s[DISP_KT], site_s[NS];
    const Geometry &g = p.g;
    const GridMap &gm = p.gm;
    const int nsite = p.nsite, nT = p.nT;
    const size_t stage_elems = (size_t)DISP_KT * NS * DISP_TC;
    C *tile = (C *)smem_raw;                                   // [2][KT][NS][TC]
    int *tinfo = (int *)(tile + 2 * stage_elems);              // [2][TC]: op | n << 2
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int k0 = blockIdx.x * DISP_KT;
    const int k = k0 + warp;
    if (threadIdx.x < DISP_KT) {
        const int kf = k0 + threadIdx.x;
        int cj = 0, ki = -1;
        if (kf < g.ncell) {
            const int f3 = kf % g.n[2], f2 = (kf / g.n[2]) % g.n[1], f1 = kf / (g.n[2] * g.n[1]);
            ki = half_index(g, f1, f2, f3, cj);
        }
        kidx_s[threadIdx.x] = ki;
        kconj_s[threadIdx.x] = cj;
    }
    if (threadIdx.x < NS) site_s[threadIdx.x] = threadIdx.x < nsite ? p.site_of[threadIdx.x] : -1;
    __syncthreads();

    const bool kvalid = k < g.ncell;
    const int kq = kvalid ? k : 0;
    const int k3 = kq % g.n[2], k2 = (kq / g.n[2]) % g.n[1], k1 = kq / (g.n[2] * g.n[1]);
    const ZoneBox zb = zone_box(g, gm, k1, k2, k3);
    const int nzk = kvalid ? zb.n[0] * zb.n[1] * zb.n[2] : 0;
    const int zbase = blockIdx.y * (32 * ZPT);
    const bool active = zbase < nzk;  // warp-uniform
    // a k of the other half of the spectrum reads the stored i^n M(-k); i^n M(k) = (-1)^n conj of it,
    // and (-1)^n c_t(Q) = c_t(-Q): such a warp runs with -Q and conjugates its sums at the end
    const bool conj = kconj_s[warp] != 0;
    const T qsign = conj ? T(-1) : T(1);

    using CP = typename CoefPair<T>::type;
    T qx[ZPT], qy[ZPT], qz[ZPT], ca[ZPT], cb[ZPT];
    CP qzp[ZPT], ccp[ZPT];
    // supercell index G of this lane's voxel j (recomputed where needed to save registers)
    auto voxel_G = [&](int j, int (&G)[3]) {
        int z = zbase + lane + 32 * j;
        if (z >= nzk) z = 0;  // computed but never stored
        const int nz23 = max(1, zb.n[1] * zb.n[2]);
        const int i1 = z / nz23, rem = z - i1 * nz23;
        const int i2 = rem / max(1, zb.n[2]), i3 = rem - i2 * max(1, zb.n[2]);
        G[0] = g.n[0] * (zb.lo[0] + i1) + k1;
        G[1] = g.n[1] * (zb.lo[1] + i2) + k2;
        G[2] = g.n[2] * (zb.lo[2] + i3) + k3;
    };
#pragma unroll
    for (int j = 0; j < ZPT; ++j) {
        int Gj[3];
        voxel_G(j, Gj);
        double Xd[3];
        x_of_G(p.gscale, g.n, Gj[0], Gj[1], Gj[2], Xd);
        qx[j] = qsign * (T)Xd[0];
        qy[j] = qsign * (T)Xd[1];
        qz[j] = qsign * (T)Xd[2];
        qzp[j] = pair_of(qz[j]);
        ca[j] = cb[j] = T(1);
        ccp[j] = pair_of(T(1));
    }
    C S[ZPT][NS];
#pragma unroll
    for (int j = 0; j < ZPT; ++j)
#pragma unroll
        for (int s = 0; s < NS; ++s) S[j][s] = mk<T>(T(0), T(0));

    // Taylor order of this CTA: the largest zone order among its voxels (all orders when no
    // per-zone table is given); its monomials are the order-Pc sub-simplex in lexicographic order
    __shared__ int pcta_s;
    int nTc = nT;
    int pzv[ZPT];
#pragma unroll
    for (int j = 0; j < ZPT; ++j) pzv[j] = 0;
    const int *tmap = nullptr, *tops = p.ops;
    if (p.pzone) {
        if (threadIdx.x == 0) pcta_s = 0;
        __syncthreads();
        int pm = 0;
#pragma unroll
        for (int j = 0; j < ZPT; ++j) {
            pzv[j] = 0;
            if (zbase + lane + 32 * j < nzk) {
                int Gj[3];
                voxel_G(j, Gj);
                const int h1 = (Gj[0] - k1) / g.n[0] - gm.Hmin[0];
                const int h2 = (Gj[1] - k2) / g.n[1] - gm.Hmin[1];
                const int h3 = (Gj[2] - k3) / g.n[2] - gm.Hmin[2];
                pzv[j] = p.pzone[((size_t)h1 * gm.nH[1] + h2) * gm.nH[2] + h3];
                pm = max(pm, pzv[j]);
            }
        }
        for (int o = 16; o > 0; o >>= 1) pm = max(pm, __shfl_xor_sync(0xffffffffu, pm, o));
        if (lane == 0) atomicMax(&pcta_s, pm);
        __syncthreads();
        const int Pc = pcta_s;
        nTc = (Pc + 1) * (Pc + 2) * (Pc + 3) / 6;
        tmap = p.sub_map + p.sub_off[Pc];
        tops = p.sub_ops + p.sub_off[Pc];
    }

    auto load_chunk = [&](int stage, int t0) {
        const int tc = min(DISP_TC, nTc - t0);
        C *dst = tile + stage * stage_elems;
        for (int idx = threadIdx.x; idx < DISP_KT * NS * DISP_TC; idx += blockDim.x) {
            const int kk = idx % DISP_KT;
            const int rest = idx / DISP_KT;
            const int tt = rest % DISP_TC, s = rest / DISP_TC;
            C *d = dst + ((size_t)kk * NS + s) * DISP_TC + tt;
            const int ki = kidx_s[kk];
            if (tt < tc && ki >= 0 && s < nsite) {
                const int t = tmap ? tmap[t0 + tt] : t0 + tt;
                cp_async<sizeof(C)>(d, p.spec + (((size_t)p.model * nsite + site_s[s]) * nT + t) * g.ncell_h + ki);
            } else {
                *d = mk<T>(T(0), T(0));
            }
        }
        for (int tt = threadIdx.x; tt < DISP_TC; tt += blockDim.x) {
            int info = 0;
            if (tt < tc) {
                const int t = tmap ? tmap[t0 + tt] : t0 + tt;
                info = tops[t0 + tt] | (p.terms[t].w << 2);
            }
            tinfo[stage * DISP_TC + tt] = info;
        }
        cp_async_commit();
    };

    const int nchunk = (nTc + DISP_TC - 1) / DISP_TC;
    load_chunk(0, 0);
    for (int c = 0; c < nchunk; ++c) {
        if (c + 1 < nchunk) load_chunk((c + 1) & 1, (c + 1) * DISP_TC);
        else cp_async_commit();
        cp_async_wait<1>();
        __syncthreads();
        if (active) {
            const int stage = c & 1;
            const int tc = min(DISP_TC, nTc - c * DISP_TC);
            const C *wt = tile + stage * stage_elems + (size_t)warp * NS * DISP_TC;
            const int *ti = tinfo + stage * DISP_TC;
            if (p.pzone) disp_chunk<T, NS, ZPT, true>(wt, ti, tc, qx, qy, qzp, pzv, ca, cb, ccp, S);
            else disp_chunk<T, NS, ZPT, false>(wt, ti, tc, qx, qy, qzp, pzv, ca, cb, ccp, S);
        }
        __syncthreads();
    }
    if (!active) return;
    if (conj) {
#pragma unroll
        for (int j = 0; j < ZPT; ++j)
#pragma unroll
            for (int s = 0; s < NS; ++s) S[j][s].y = -S[j][s].y;
    }

    // epilogue: F = sum_mu b f(|G|) exp(iG.r_mu) S_mu, minus <F(H)> at k = 0, I = |F|^2 norm
#pragma unroll
    for (int j = 0; j < ZPT; ++j) {
        const int z = zbase + lane + 32 * j;
        if (z >= nzk) continue;
        int Gj[3];
        voxel_G(j, Gj);
        const int G1 = Gj[0], G2 = Gj[1], G3 = Gj[2];
        double Qd[3];
        q_of_G(p.recip, g.n, G1, G2, G3, Qd);
        const T q2 = (T)(Qd[0] * Qd[0] + Qd[1] * Qd[1] + Qd[2] * Qd[2]);
        const T s2 = q2 * (T)(1.0 / (FOUR_PI_D * FOUR_PI_D));
        const int H1 = (G1 - k1) / g.n[0], H2 = (G2 - k2) / g.n[1], H3 = (G3 - k3) / g.n[2];
        const int h1 = H1 - gm.Hmin[0], h2 = H2 - gm.Hmin[1], h3 = H3 - gm.Hmin[2];
        C F = mk<T>(T(0), T(0)), part = mk<T>(T(0), T(0));
        int cls = 0;
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            if (s < nsite) {
                const int site = site_s[s];
                const C *tH = p.phH + (size_t)site * 3 * p.nHmax;
                const C *tk = p.phk + (size_t)site * 3 * p.nmax;
                C ph = cmul(cmul(tH[h1], tH[p.nHmax + h2]), tH[2 * p.nHmax + h3]);
                ph = cmul(ph, cmul(cmul(tk[k1], tk[p.nmax + k2]), tk[2 * p.nmax + k3]));
                ph = cscale(ph, p.scat[site]);
                cfma(part, ph, S[j][s]);
                if (s + 1 == p.ff.cls_end[cls]) {
                    const T f = form_factor<T>(p.ff.cls_kind[cls], p.ff.cls_coef[cls], s2);
                    F.x = fma(f, part.x, F.x);
                    F.y = fma(f, part.y, F.y);
                    part = mk<T>(T(0), T(0));
                    ++cls;
                }
            }
        }
        if (p.diffuse && k1 == 0 && k2 == 0 && k3 == 0) {
            const C b = p.bragg[((size_t)h1 * gm.nH[1] + h2) * gm.nH[2] + h3];
            F = csub(F, b);
        }
        const T I = F.x * F.x + F.y * F.y;
        const size_t v = ((size_t)(G1 - gm.g0[0]) * gm.cnt[1] + (G2 - gm.g0[1])) * gm.cnt[2] + (G3 - gm.g0[2]);
        const T val = p.norm * I;
        p.out[v] = p.accumulate ? p.out[v] + val : val;
        if (p.Fout) p.Fout[(size_t)p.model * gm.cnt[0] * gm.cnt[1] * gm.cnt[2] + v] = F;
    }
}

template <typename T, int NS, int ZPT, int MINB> static void launch_disp(const RecombParams<T> &p, cudaStream_t s) {
    using C = c_t<T>;
    // the largest per-k zone box bounds the zone chunks
    int nzmax = 1;
    for (int a = 0; a < 3; ++a) nzmax *= (p.gm.cnt[a] + p.g.n[a] - 1) / p.g.n[a] + 1;
    dim3 grid((p.g.ncell + DISP_KT - 1) / DISP_KT, (nzmax + 32 * ZPT - 1) / (32 * ZPT));
    const size_t sm = 2 * (size_t)DISP_KT * NS * DISP_TC * sizeof(C) + 2 * DISP_TC * sizeof(int);
    if (sm > 48 * 1024)
        cudaFuncSetAttribute(k_recomb_disp<T, NS, ZPT, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_recomb_disp<T, NS, ZPT, MINB><<<grid, DISP_KT * 32, sm, s>>>(p);
    count_launches(1);
}

// sites per thread: exact for 1..8 sites (no idle rows), 16 rows (zero-padded) above
template <typename T> void recombine_disp(const RecombParams<T> &p, cudaStream_t s) {
    constexpr bool dbl = sizeof(T) == 8;
    switch (p.nsite) {
        case 1: launch_disp<T, 1, dbl ? 2 : 4, 2>(p, s); break;
        case 2: launch_disp<T, 2, dbl ? 2 : 4, 2>(p, s); break;
        case 3: launch_disp<T, 3, dbl ? 2 : 4, 2>(p, s); break;
        case 4: launch_disp<T, 4, dbl ? 2 : 4, 2>(p, s); break;
        case 5: launch_disp<T, 5, dbl ? 2 : 4, dbl ? 1 : 2>(p, s); break;
        case 6: launch_disp<T, 6, 2, dbl ? 1 : 2>(p, s); break;
        case 7: launch_disp<T, 7, 2, dbl ? 1 : 2>(p, s); break;
        case 8: launch_disp<T, 8, 2, dbl ? 1 : 2>(p, s); break;
        default: launch_disp<T, 16, dbl ? 1 : 2, 1>(p, s); break;
    }
}

// <F(H)> of Eq. bragg_sf_disp: even orders of the k = 0 transforms averaged over supercells
template <typename T>
__global__ void k_avg0(int nmodels, int nsite, int nT, int ncell_h, const int4 *terms, const c_t<T> *spec,
                       c_t<T> *avg0) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= nsite * nT) return;
    const int t = idx % nT;
    c_t<T> acc = mk<T>(T(0), T(0));
    if ((terms[t].w & 1) == 0)
        for (int m = 0; m < nmodels; ++m) acc = cadd(acc, spec[((size_t)m * nsite * nT + idx) * ncell_h]);
    avg0[idx] = cscale(acc, T(1) / T(nmodels));
}

// <F(H)> per zone H (Eq. bragg_sf_disp with the Taylor series of <exp(iQ.u)>): a warp per zone.
// Lane 0 tabulates the zone's powers x_a^e (e <= P) of the scaled coefficient variables in shared
// memory; the lanes split each site's monomials, x1^a x2^b x3^c times the site's mean coefficient,
// and a warp reduction gives the site sum; phases and the class form factors as in Eq. sf.
template <typename T>
__global__ void __launch_bounds__(256) k_bragg_disp(RecombParams<T> p, const c_t<T> *avg0, c_t<T> *bragg_out, int P) {
    using C = c_t<T>;
    extern __shared__ double bragg_pw[];
    const GridMap &gm = p.gm;
    const int nz = gm.nH[0] * gm.nH[1] * gm.nH[2];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int z = blockIdx.x * 8 + warp;
    if (z >= nz) return;   // whole warps only: no block-wide barrier below
    const int P1 = P + 1;
    double *pw = bragg_pw + warp * 3 * P1;
    const int h3 = z % gm.nH[2], h2 = (z / gm.nH[2]) % gm.nH[1], h1 = z / (gm.nH[2] * gm.nH[1]);
    const int G1 = p.g.n[0] * (gm.Hmin[0] + h1), G2 = p.g.n[1] * (gm.Hmin[1] + h2), G3 = p.g.n[2] * (gm.Hmin[2] + h3);
    double Qd[3], Xd[3];
    q_of_G(p.recip, p.g.n, G1, G2, G3, Qd);
    x_of_G(p.gscale, p.g.n, G1, G2, G3, Xd);
    if (lane < 3) {
        double v = 1.0;
        for (int e = 0; e <= P; ++e) {
            pw[lane * P1 + e] = v;
            v *= Xd[lane];
        }
    }
    __syncwarp();
    const T q2 = (T)(Qd[0] * Qd[0] + Qd[1] * Qd[1] + Qd[2] * Qd[2]);
    const T s2 = q2 * (T)(1.0 / (FOUR_PI_D * FOUR_PI_D));
    C F = mk<T>(T(0), T(0)), part = mk<T>(T(0), T(0));
    int cls = 0;
    const int pz = p.pzone ? p.pzone[z] : 1 << 30;  // the zone's Taylor order
    for (int s = 0; s < p.nsite; ++s) {
        const int site = p.site_of[s];
        T sx = T(0), sy = T(0);
        for (int t = lane; t < p.nT; t += 32) {
            const int4 tm = p.terms[t];
            if (tm.w > pz) continue;
            const T mono = (T)(pw[tm.x] * pw[P1 + tm.y] * pw[2 * P1 + tm.z]);
            const C m = avg0[(size_t)site * p.nT + t];
            sx = fma(mono, m.x, sx);
            sy = fma(mono, m.y, sy);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            sx += __shfl_xor_sync(0xffffffffu, sx, o);
            sy += __shfl_xor_sync(0xffffffffu, sy, o);
        }
        const C S = mk<T>(sx, sy);
        const C *tH = p.phH + (size_t)site * 3 * p.nHmax;
        C ph = cmul(cmul(tH[h1], tH[p.nHmax + h2]), tH[2 * p.nHmax + h3]);
        ph = cscale(ph, p.scat[site]);
        part = cadd(part, cmul(ph, S));
        if (s + 1 == p.ff.cls_end[cls]) {
            const T f = form_factor<T>(p.ff.cls_kind[cls], p.ff.cls_coef[cls], s2);
            F = cadd(F, cscale(part, f));
            part = mk<T>(T(0), T(0));
            ++cls;
        }
    }
    if (lane == 0) bragg_out[z] = F;
}

template <typename T>
void displacive_bragg(const RecombParams<T> &p, const int4 *terms, c_t<T> *avg0, c_t<T> *bragg, cudaStream_t s) {
    const int n0 = p.nsite * p.nT;
    k_avg0<T><<<(n0 + 255) / 256, 256, 0, s>>>(p.nmodels, p.nsite, p.nT, p.g.ncell_h, terms, p.spec, avg0);
    const int nz = p.gm.nH[0] * p.gm.nH[1] * p.gm.nH[2];
    int P = 0;   // the order of the nT monomials: (P + 1)(P + 2)(P + 3) / 6 = nT
    while ((P + 1) * (P + 2) * (P + 3) / 6 < p.nT) ++P;
    const size_t sm = (size_t)8 * 3 * (P + 1) * sizeof(double);
    if (sm > 48 * 1024) cudaFuncSetAttribute(k_bragg_disp<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_bragg_disp<T><<<(nz + 7) / 8, 256, sm, s>>>(p, avg0, bragg, P);
    count_launches(2);
}

#define DS_INST(T)                                                                                          \
    template void make_site_tables<T>(const Geometry &, const GridMap &, int, const double *, c_t<T> *,     \
                                      c_t<T> *, int, int, cudaStream_t);                                    \
    template void make_powers<T>(const Geometry &, int, int, int, const double *, const double *, const float *, T *, \
                                 cudaStream_t);                                                             \
    template void recombine_cm<T>(const RecombParams<T> &, cudaStream_t);                                   \
    template void recombine_disp<T>(const RecombParams<T> &, cudaStream_t);                                 \
    template void displacive_bragg<T>(const RecombParams<T> &, const int4 *, c_t<T> *, c_t<T> *, cudaStream_t);
DS_INST(float)
DS_INST(double)

}  // namespace ds
