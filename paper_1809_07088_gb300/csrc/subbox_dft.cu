// Method of sub-boxes by direct summation over origins (Section V A), at arbitrary wavevectors,
// and the Debye-Waller factor T_mu(Q) of Eq. dw.
//
// Sub-boxes.  For every origin (m, o) -- the lattice point o of supercell m, from a list the
// caller draws at random (the original random-origin variant) or every lattice point of every
// supercell (the every-lattice-point variant) -- the n_sb^3 cells o + d, d in [0, n_sb)^3, form
// a box with open boundaries:
//     F_o(Q) = sum_d exp(2 pi i Q.d) sum_mu phi_mu(Q) [a_{(o+d) mod n, mu}(Q) - abar_mu(Q)],
//     phi_mu(Q) = b_mu f_mu(|Q|) exp(2 pi i Q.r_mu),
// with a = delta (occupancy), M (moment, three components) or delta exp(i Q.u) (displacement,
// the exact exponential: no Taylor expansion), and abar = 0 (TOTAL) or the site mean c_mu,
// <M>_mu or <delta cos(Q.u)>_mu (DIFFUSE; the last is the Debye-Waller factor below), and
//     I(Q) = sum_o |F_o(Q)|^2 / (norigin nsite n_sb^3)     (magnetic: C |F_o,perp|^2).
// The common phase exp(2 pi i Q.o) of a box drops out of |F_o|^2.
//
// One thread per Q point.  A block walks its share of the origins; the atoms of each box are
// staged in shared memory as float4 (delta / M / (u, delta)) and read by all lanes at once.  The
// per-Q constants -- phi_mu, the diffuse constant sum_mu phi_mu abar_mu and the one-cell steps
// of Q.d -- are formed in FP64 and kept in registers in the working precision.  Each block
// writes its partial sum over its origin chunk; a second kernel adds the chunks in a fixed order.
//
// Debye-Waller factor.  T_mu(Q) = (1/(nmodels n1 n2 n3)) sum_{m,R} w cos(Q.u_{m,R,mu}), w = 1
// or the occupancy delta: the even part of Eq. dw (its odd orders in Q.u average to zero over
// the ensemble, Section III C, as for <F(H)>).  One thread per (Q, site), the displacements of
// that site staged in shared memory.  It is the per-site factor of Eq. mag_sf (the magnetic +
// displacive coupling) and the site mean of the displacive sub-box.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "api_internal.h"

using namespace ds;

namespace {

constexpr int SB_THREADS = 128;
constexpr int SB_STAGE = 2048;   // atoms staged per pass (float4: 32 KB)
constexpr int DW_THREADS = 128;
constexpr int DW_STAGE = 1024;
enum { SB_OCC = 0, SB_SPIN = 1, SB_DISP = 2 };

// per-site constants of the sub-box sum (FP64, built on the host)
struct SbSite {
    double r[3];
    double b;
    double coef[9];
    int kind;
    int pad;
};

template <typename T> struct SbParams {
    int nsite, nsb, n1, n2, n3, ncell;
    int diffuse;
    const SbSite *site;    // [nsite]
    const uint8_t *occ;    // [model][site][cell]: occupancy; displacive weights (may be null)
    const float *vec;      // moments or displacements [model][site][cell][3]
    const double *mean;    // DIFFUSE: c_mu [site] or <M>_mu [site][3]
    const T *dw;           // DIFFUSE displacive: <delta cos(Q.u)>_mu [site][npts]
    const double *hkl;     // [npts][3] r.l.u.
    long long npts;
    const int4 *origins;   // (model, o1, o2, o3)
    long long norigin, per_chunk;
    double recip[9];       // a*, b*, c* rows (1/A, 2 pi included)
    T *partial;            // [chunk][npts]
};

// Phases are carried in cycles (Q.x / 2 pi) and brought to [-1/2, 1/2] by subtracting the
// nearest integer before the sine and cosine, where the fast FP32 __sincosf / __cosf are
// accurate; FP64 uses sincospi / cospi.
// x minus its nearest integer.  FP32: adding and subtracting 1.5 * 2^23 rounds |x| < 2^22 to
// the nearest integer on the FMA pipe (rintf would take a slot of the SFU/conversion pipe that
// the sine and cosine need); phases here are a few cycles.
__device__ __forceinline__ double frac_w(double x) { return x - rint(x); }
__device__ __forceinline__ float frac_w(float x) {
    const float r = __fsub_rn(__fadd_rn(x, 12582912.0f), 12582912.0f);
    return __fsub_rn(x, r);
}
// cos 2 pi t for a phase t in cycles (reduced to [-1/2, 1/2] first)
__device__ __forceinline__ double cos_cycles(double t) { return cospi(2.0 * frac_w(t)); }
__device__ __forceinline__ float cos_cycles(float t) { return __cosf(frac_w(t) * 6.283185307179586f); }
// (cos 2 pi r, sin 2 pi r) for |r| <= 1/2
__device__ __forceinline__ void sincos_cycles(double r, double &c, double &s) { sincospi(2.0 * r, &s, &c); }
__device__ __forceinline__ void sincos_cycles(float r, float &c, float &s) { __sincosf(r * 6.283185307179586f, &s, &c); }
// S += phi (c + i s) = phi c + (i phi) s: two paired FP32 multiply-adds
__device__ __forceinline__ void cexp_acc(float2 &S, float2 phi, float2 iphi, float c, float s) {
    S = __ffma2_rn(phi, make_float2(c, c), S);
    S = __ffma2_rn(iphi, make_float2(s, s), S);
}
__device__ __forceinline__ void cexp_acc(double2 &S, double2 phi, double2 iphi, double c, double s) {
    S.x = fma(phi.x, c, S.x);
    S.x = fma(iphi.x, s, S.x);
    S.y = fma(phi.y, c, S.y);
    S.y = fma(iphi.y, s, S.y);
}

// Occupational and magnetic boxes: per cell, the site sum sum_mu phi_mu (a - abar) times the
// cell phase exp(2 pi i Q.d), advanced by one complex multiply per cell.
template <typename T, int KIND, int MAXS>
__global__ void __launch_bounds__(SB_THREADS) k_subbox_dft(const __grid_constant__ SbParams<T> p) {
    using C = c_t<T>;
    constexpr int NC = KIND == SB_SPIN ? 3 : 1;
    __shared__ float4 stage[SB_STAGE];
    const long long q = (long long)blockIdx.x * SB_THREADS + threadIdx.x;
    const bool live = q < p.npts;
    const long long qq = live ? q : p.npts - 1;  // idle lanes repeat the last point (stores skipped)
    const int nsite = p.nsite, nsb = p.nsb;

    // per-point constants in FP64
    const double h[3] = {p.hkl[3 * qq], p.hkl[3 * qq + 1], p.hkl[3 * qq + 2]};
    double Qd[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) Qd[a] = h[0] * p.recip[a] + h[1] * p.recip[3 + a] + h[2] * p.recip[6 + a];
    const double q2d = Qd[0] * Qd[0] + Qd[1] * Qd[1] + Qd[2] * Qd[2];
    const double s2 = q2d / (FOUR_PI_D * FOUR_PI_D);
    C phi[MAXS];
    double Kd[NC][2];
#pragma unroll
    for (int c = 0; c < NC; ++c) Kd[c][0] = Kd[c][1] = 0.0;
#pragma unroll
    for (int s = 0; s < MAXS; ++s) {
        phi[s] = mk<T>(T(0), T(0));
        if (s < nsite) {
            const SbSite &S = p.site[s];
            const double f = S.b * form_factor<double>(S.kind, S.coef, s2);
            double t = h[0] * S.r[0] + h[1] * S.r[1] + h[2] * S.r[2];
            t -= rint(t);
            double sn, cs;
            sincospi(2.0 * t, &sn, &cs);
            const double pr = f * cs, pi = f * sn;
            phi[s] = mk<T>((T)pr, (T)pi);
            if (p.diffuse) {
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    double abar;
                    if (KIND == SB_OCC) abar = p.mean[s];
                    else abar = p.mean[3 * s + c];
                    Kd[c][0] += pr * abar;
                    Kd[c][1] += pi * abar;
                }
            }
        }
    }
    C K[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) K[c] = mk<T>((T)Kd[c][0], (T)Kd[c][1]);
    C e[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        double sn, cs;
        sincospi(2.0 * (h[a] - rint(h[a])), &sn, &cs);
        e[a] = mk<T>((T)cs, (T)sn);
    }
    const T Qx = (T)Qd[0], Qy = (T)Qd[1], Qz = (T)Qd[2];

    T acc = T(0);
    const long long o0 = (long long)blockIdx.y * p.per_chunk;
    const long long o1 = min(p.norigin, o0 + p.per_chunk);
    const int nbox = nsb * nsb * nsb;
    const int cps = max(1, SB_STAGE / nsite);  // cells per staging pass
    for (long long oi = o0; oi < o1; ++oi) {
        const int4 og = p.origins[oi];
        C F[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) F[c] = mk<T>(T(0), T(0));
        C P1 = mk<T>(T(1), T(0)), P12 = P1, P = P1;
        int d2 = 0, d3 = 0;
        for (int c0 = 0; c0 < nbox; c0 += cps) {
            const int ncs = min(cps, nbox - c0);
            __syncthreads();
            for (int i = threadIdx.x; i < ncs * nsite; i += SB_THREADS) {
                const int cc = i / nsite, s = i - cc * nsite;
                const int c = c0 + cc;
                const int e1 = c / (nsb * nsb), e2 = (c / nsb) % nsb, e3 = c % nsb;
                int w1 = og.y + e1, w2 = og.z + e2, w3 = og.w + e3;  // o < n and d < n_sb <= n
                if (w1 >= p.n1) w1 -= p.n1;
                if (w2 >= p.n2) w2 -= p.n2;
                if (w3 >= p.n3) w3 -= p.n3;
                const size_t base = ((size_t)og.x * nsite + s) * p.ncell + ((size_t)w1 * p.n2 + w2) * p.n3 + w3;
                float4 v;
                if (KIND == SB_OCC) {
                    v = make_float4((float)p.occ[base], 0.f, 0.f, 0.f);
                } else {
                    v.x = p.vec[3 * base];
                    v.y = p.vec[3 * base + 1];
                    v.z = p.vec[3 * base + 2];
                    v.w = 0.f;
                }
                stage[i] = v;
            }
            __syncthreads();
            for (int cc = 0; cc < ncs; ++cc) {
                C part[NC], alt = mk<T>(T(0), T(0));  // alt: odd sites of the occupancy sum
#pragma unroll
                for (int c = 0; c < NC; ++c) part[c] = mk<T>(-K[c].x, -K[c].y);
                const float4 *at = stage + cc * nsite;
#pragma unroll
                for (int s = 0; s < MAXS; ++s) {
                    if (s < nsite) {
                        const float4 v = at[s];
                        if (KIND == SB_OCC) {
                            C &a = (s & 1) ? alt : part[0];
                            a.x = fma(phi[s].x, (T)v.x, a.x);
                            a.y = fma(phi[s].y, (T)v.x, a.y);
                        } else {
                            const T m3[3] = {(T)v.x, (T)v.y, (T)v.z};
#pragma unroll
                            for (int c = 0; c < NC; ++c) {
                                part[c].x = fma(phi[s].x, m3[c], part[c].x);
                                part[c].y = fma(phi[s].y, m3[c], part[c].y);
                            }
                        }
                    }
                }
                if (KIND == SB_OCC) part[0] = cadd(part[0], alt);
#pragma unroll
                for (int c = 0; c < NC; ++c) cfma(F[c], P, part[c]);
                // the next cell of the box (d3 fastest)
                if (++d3 == nsb) {
                    d3 = 0;
                    if (++d2 == nsb) {
                        d2 = 0;
                        P1 = cmul(P1, e[0]);
                        P12 = P1;
                    } else {
                        P12 = cmul(P12, e[1]);
                    }
                    P = P12;
                } else {
                    P = cmul(P, e[2]);
                }
            }
        }
        T tot = T(0);
#pragma unroll
        for (int c = 0; c < NC; ++c) tot += F[c].x * F[c].x + F[c].y * F[c].y;
        if (KIND == SB_SPIN) {
            const T q2 = Qx * Qx + Qy * Qy + Qz * Qz;
            if (q2 > T(0)) {
                const T pr = Qx * F[0].x + Qy * F[1].x + Qz * F[2].x;
                const T pi = Qx * F[0].y + Qy * F[1].y + Qz * F[2].y;
                tot -= (pr * pr + pi * pi) / q2;
            } else {
                tot *= T(2) / T(3);
            }
        }
        acc += tot;
    }
    if (live) p.partial[(size_t)blockIdx.y * p.npts + q] = acc;
}

// Displacive boxes: the cell offset d is folded into each atom's phase, in cycles, and the
// site factor phi_mu is applied once per box:
//     F_o = sum_mu phi_mu sum_d w exp(2 pi i (Q.d + Q.u / 2 pi)) - K B,
// Q.d kept reduced to [-1/2, 1/2] and advanced by one add per cell, so that each atom costs
// three multiply-adds, one reduction, one sincos and two adds into its site's (cos, sin) sums;
// K = sum_mu phi_mu <w cos(Q.u)>_mu and B = sum_d exp(2 pi i Q.d) (the box's geometric series,
// FP64) carry the DIFFUSE subtraction.  EXACT: nsite == MAXS (no per-site guard).
template <typename T, int MAXS, bool EXACT, bool WEIGHTED>
__global__ void __launch_bounds__(SB_THREADS) k_subbox_dft_disp(const __grid_constant__ SbParams<T> p) {
    using C = c_t<T>;
    __shared__ float4 stage[SB_STAGE];
    const long long q = (long long)blockIdx.x * SB_THREADS + threadIdx.x;
    const bool live = q < p.npts;
    const long long qq = live ? q : p.npts - 1;
    const int nsite = EXACT ? MAXS : p.nsite, nsb = p.nsb;
    const double h[3] = {p.hkl[3 * qq], p.hkl[3 * qq + 1], p.hkl[3 * qq + 2]};
    double Qd[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) Qd[a] = h[0] * p.recip[a] + h[1] * p.recip[3 + a] + h[2] * p.recip[6 + a];
    const double s2 = (Qd[0] * Qd[0] + Qd[1] * Qd[1] + Qd[2] * Qd[2]) / (FOUR_PI_D * FOUR_PI_D);
    C phi[MAXS];
    double Kr = 0.0, Ki = 0.0;
#pragma unroll
    for (int s = 0; s < MAXS; ++s) {
        phi[s] = mk<T>(T(0), T(0));
        if (s < nsite) {
            const SbSite &S = p.site[s];
            const double f = S.b * form_factor<double>(S.kind, S.coef, s2);
            double sn, cs;
            sincospi(2.0 * frac_w(h[0] * S.r[0] + h[1] * S.r[1] + h[2] * S.r[2]), &sn, &cs);
            phi[s] = mk<T>((T)(f * cs), (T)(f * sn));
            if (p.diffuse) {
                const double t = (double)p.dw[(size_t)s * p.npts + qq];
                Kr += f * cs * t;
                Ki += f * sn * t;
            }
        }
    }
    // K B: the box sum of the site-mean amplitudes
    double Br = 1.0, Bi = 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        double sr = 0.0, si = 0.0;
        const double fa = frac_w(h[a]);
        for (int d = 0; d < nsb; ++d) {
            double sn, cs;
            sincospi(2.0 * frac_w(fa * d), &sn, &cs);
            sr += cs;
            si += sn;
        }
        const double tr = Br * sr - Bi * si;
        Bi = Br * si + Bi * sr;
        Br = tr;
    }
    const C KB = mk<T>((T)(Kr * Br - Ki * Bi), (T)(Kr * Bi + Ki * Br));
    const T f1 = (T)frac_w(h[0]), f2 = (T)frac_w(h[1]), f3 = (T)frac_w(h[2]);
    const double inv2pi = 1.0 / TWO_PI_D;
    const T Qx = (T)(Qd[0] * inv2pi), Qy = (T)(Qd[1] * inv2pi), Qz = (T)(Qd[2] * inv2pi);  // cycles per A

    T acc = T(0);
    const long long o0 = (long long)blockIdx.y * p.per_chunk;
    const long long o1 = min(p.norigin, o0 + p.per_chunk);
    const int nbox = nsb * nsb * nsb;
    const int cps = max(1, SB_STAGE / nsite);
    for (long long oi = o0; oi < o1; ++oi) {
        const int4 og = p.origins[oi];
        T Ac[MAXS], As[MAXS];  // per site: sum over the box of w cos, w sin
#pragma unroll
        for (int s = 0; s < MAXS; ++s) Ac[s] = As[s] = T(0);
        T c1 = T(0), c12 = T(0), c = T(0);  // Q.d in cycles, reduced
        int d2 = 0, d3 = 0;
        for (int c0 = 0; c0 < nbox; c0 += cps) {
            const int ncs = min(cps, nbox - c0);
            __syncthreads();
            for (int i = threadIdx.x; i < ncs * nsite; i += SB_THREADS) {
                const int cc = i / nsite, s = i - cc * nsite;
                const int cl = c0 + cc;
                const int e1 = cl / (nsb * nsb), e2 = (cl / nsb) % nsb, e3 = cl % nsb;
                int w1 = og.y + e1, w2 = og.z + e2, w3 = og.w + e3;  // o < n and d < n_sb <= n
                if (w1 >= p.n1) w1 -= p.n1;
                if (w2 >= p.n2) w2 -= p.n2;
                if (w3 >= p.n3) w3 -= p.n3;
                const size_t base = ((size_t)og.x * nsite + s) * p.ncell + ((size_t)w1 * p.n2 + w2) * p.n3 + w3;
                stage[i] = make_float4(p.vec[3 * base], p.vec[3 * base + 1], p.vec[3 * base + 2],
                                       WEIGHTED ? (float)p.occ[base] : 1.f);
            }
            __syncthreads();
            for (int cc = 0; cc < ncs; ++cc) {
                const float4 *at = stage + cc * nsite;
#pragma unroll
                for (int s = 0; s < MAXS; ++s) {
                    if (EXACT || s < nsite) {
                        const float4 v = at[s];
                        const T t = fma(Qx, (T)v.x, fma(Qy, (T)v.y, fma(Qz, (T)v.z, c)));
                        T cs, sn;
                        sincos_cycles(frac_w(t), cs, sn);
                        if (WEIGHTED) {
                            Ac[s] = fma((T)v.w, cs, Ac[s]);
                            As[s] = fma((T)v.w, sn, As[s]);
                        } else {
                            Ac[s] += cs;
                            As[s] += sn;
                        }
                    }
                }
                if (++d3 == nsb) {
                    d3 = 0;
                    if (++d2 == nsb) {
                        d2 = 0;
                        c1 = frac_w(c1 + f1);
                        c12 = c1;
                    } else {
                        c12 = frac_w(c12 + f2);
                    }
                    c = c12;
                } else {
                    c = frac_w(c + f3);
                }
            }
        }
        C F = mk<T>(-KB.x, -KB.y);
#pragma unroll
        for (int s = 0; s < MAXS; ++s) {
            F.x = fma(phi[s].x, Ac[s], fma(-phi[s].y, As[s], F.x));
            F.y = fma(phi[s].x, As[s], fma(phi[s].y, Ac[s], F.y));
        }
        acc += F.x * F.x + F.y * F.y;
    }
    if (live) p.partial[(size_t)blockIdx.y * p.npts + q] = acc;
}

template <typename T>
__global__ void k_sum_chunks(const T *__restrict__ partial, long long npts, int nchunk, double norm,
                             T *__restrict__ out) {
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < npts; q += (long long)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int c = 0; c < nchunk; ++c) s += (double)partial[(size_t)c * npts + q];
        out[q] = (T)(s * norm);
    }
}

template <typename T> using SbKernel = void (*)(SbParams<T>);

template <typename T, bool W> SbKernel<T> disp_kernel(int nsite) {
    if constexpr (sizeof(T) == 4) {  // the FP32 path holds exactly nsite sites for nsite <= 8
        switch (nsite) {
        case 1: return k_subbox_dft_disp<T, 1, true, W>;
        case 2: return k_subbox_dft_disp<T, 2, true, W>;
        case 3: return k_subbox_dft_disp<T, 3, true, W>;
        case 4: return k_subbox_dft_disp<T, 4, true, W>;
        case 5: return k_subbox_dft_disp<T, 5, true, W>;
        case 6: return k_subbox_dft_disp<T, 6, true, W>;
        case 7: return k_subbox_dft_disp<T, 7, true, W>;
        case 8: return k_subbox_dft_disp<T, 8, true, W>;
        default: break;
        }
    } else {
        if (nsite <= 4) return k_subbox_dft_disp<T, 4, false, W>;
        if (nsite <= 8) return k_subbox_dft_disp<T, 8, false, W>;
    }
    return k_subbox_dft_disp<T, 16, false, W>;
}
template <typename T, int KIND> SbKernel<T> site_sum_kernel(int nsite) {
    if (nsite <= 4) return k_subbox_dft<T, KIND, 4>;
    if (nsite <= 8) return k_subbox_dft<T, KIND, 8>;
    return k_subbox_dft<T, KIND, 16>;
}
template <typename T> SbKernel<T> subbox_kernel(int kind, int nsite, bool weighted) {
    if (kind == SB_DISP) return weighted ? disp_kernel<T, true>(nsite) : disp_kernel<T, false>(nsite);
    return kind == SB_OCC ? site_sum_kernel<T, SB_OCC>(nsite) : site_sum_kernel<T, SB_SPIN>(nsite);
}

// Origins per block: every block does the same work (per_chunk origins x 128 points), so the
// launch takes ceil(blocks / resident) equal waves; the smallest chunk count whose wave
// efficiency is within 3 % of the best (with at least 8 origins per chunk) is chosen.
long long origin_chunks(long long norigin, long long pblocks, long long resident) {
    const long long minper = std::min<long long>(8, norigin);
    double best = 0.0;
    std::vector<std::pair<double, long long>> cand;
    for (long long c = 1; c <= std::min<long long>(norigin, 65535); ++c) {
        const long long per = (norigin + c - 1) / c;
        if (per < minper) break;
        const long long cc = (norigin + per - 1) / per;
        const long long waves = (pblocks * cc + resident - 1) / resident;
        const double eff = (double)norigin * pblocks / ((double)waves * resident * per);
        cand.push_back({eff, per});
        best = std::max(best, eff);
    }
    for (auto &e : cand)
        if (e.first >= 0.97 * best) return e.second;
    return norigin;
}

// ---------------------------------------------------------------------------------------------
// Debye-Waller factor
// ---------------------------------------------------------------------------------------------

template <typename T> struct DwParams {
    int nsite, ncell, nmodels;
    const float *disp;      // [model][site][cell][3]
    const uint8_t *occ;     // weights (null: 1)
    // points: hkl [npts][3] (r.l.u.); grid: G_a = g0_a + i_a, Q = sum_a G_a qstep_a (rows kernel)
    const double *hkl;
    int g0[3], cnt[3];
    double qstep[9];
    double recip[9];
    long long npts;
    long long site_stride, pt_stride;
    T *out;
};

template <typename T>
__global__ void __launch_bounds__(DW_THREADS) k_debye_waller(const __grid_constant__ DwParams<T> p) {
    __shared__ float4 stage[DW_STAGE];
    const int s = blockIdx.y;
    const long long q = (long long)blockIdx.x * DW_THREADS + threadIdx.x;
    const bool live = q < p.npts;
    const long long qq = live ? q : p.npts - 1;
    double Qd[3];
    const double h0 = p.hkl[3 * qq], h1 = p.hkl[3 * qq + 1], h2 = p.hkl[3 * qq + 2];
#pragma unroll
    for (int a = 0; a < 3; ++a) Qd[a] = h0 * p.recip[a] + h1 * p.recip[3 + a] + h2 * p.recip[6 + a];
    const double inv2pi = 1.0 / TWO_PI_D;
    const T Qx = (T)(Qd[0] * inv2pi), Qy = (T)(Qd[1] * inv2pi), Qz = (T)(Qd[2] * inv2pi);  // cycles per A
    const long long nsamp = (long long)p.nmodels * p.ncell;
    T acc0 = T(0), acc1 = T(0);
    for (long long j0 = 0; j0 < nsamp; j0 += DW_STAGE) {
        const int n = (int)min((long long)DW_STAGE, nsamp - j0);
        __syncthreads();
        for (int i = threadIdx.x; i < n; i += DW_THREADS) {
            const long long j = j0 + i;
            const long long m = j / p.ncell, cell = j - m * p.ncell;
            const size_t base = ((size_t)m * p.nsite + s) * p.ncell + cell;
            stage[i] = make_float4(p.disp[3 * base], p.disp[3 * base + 1], p.disp[3 * base + 2],
                                   p.occ ? (float)p.occ[base] : 1.f);
        }
        __syncthreads();
        int i = 0;
        for (; i + 1 < n; i += 2) {
            const float4 a = stage[i], b = stage[i + 1];
            acc0 = fma((T)a.w, cos_cycles(fma(Qx, (T)a.x, fma(Qy, (T)a.y, Qz * (T)a.z))), acc0);
            acc1 = fma((T)b.w, cos_cycles(fma(Qx, (T)b.x, fma(Qy, (T)b.y, Qz * (T)b.z))), acc1);
        }
        if (i < n) {
            const float4 a = stage[i];
            acc0 = fma((T)a.w, cos_cycles(fma(Qx, (T)a.x, fma(Qy, (T)a.y, Qz * (T)a.z))), acc0);
        }
    }
    if (live) p.out[(size_t)s * p.site_stride + (size_t)q * p.pt_stride] = (acc0 + acc1) / (T)nsamp;
}

// On a grid, one thread takes VPT consecutive voxels of a row along the last axis: per lattice
// point it forms z = exp(2 pi i Q_0.u) and the one-voxel step w = exp(2 pi i c*.u / n3) (two
// sincos), then walks the row by z <- z w (four multiply-adds per voxel, no SFU operation).
template <typename T, int VPT>
__global__ void __launch_bounds__(DW_THREADS) k_debye_waller_rows(const __grid_constant__ DwParams<T> p) {
    __shared__ float4 stage[DW_STAGE];
    const int s = blockIdx.y;
    const int nseg = (p.cnt[2] + VPT - 1) / VPT;
    const long long nwork = (long long)p.cnt[0] * p.cnt[1] * nseg;
    const long long wi = (long long)blockIdx.x * DW_THREADS + threadIdx.x;
    const bool live = wi < nwork;
    const long long ww = live ? wi : nwork - 1;
    const long long row = ww / nseg;
    const int i2_0 = (int)(ww - row * nseg) * VPT;
    const int i1 = (int)(row % p.cnt[1]), i0 = (int)(row / p.cnt[1]);
    const double G[3] = {(double)(p.g0[0] + i0), (double)(p.g0[1] + i1), (double)(p.g0[2] + i2_0)};
    const double inv2pi = 1.0 / TWO_PI_D;
    T Q0[3], St[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        Q0[a] = (T)((G[0] * p.qstep[a] + G[1] * p.qstep[3 + a] + G[2] * p.qstep[6 + a]) * inv2pi);
        St[a] = (T)(p.qstep[6 + a] * inv2pi);
    }
    const long long nsamp = (long long)p.nmodels * p.ncell;
    T acc[VPT];
#pragma unroll
    for (int j = 0; j < VPT; ++j) acc[j] = T(0);
    for (long long j0 = 0; j0 < nsamp; j0 += DW_STAGE) {
        const int n = (int)min((long long)DW_STAGE, nsamp - j0);
        __syncthreads();
        for (int i = threadIdx.x; i < n; i += DW_THREADS) {
            const long long j = j0 + i;
            const long long m = j / p.ncell, cell = j - m * p.ncell;
            const size_t base = ((size_t)m * p.nsite + s) * p.ncell + cell;
            stage[i] = make_float4(p.disp[3 * base], p.disp[3 * base + 1], p.disp[3 * base + 2],
                                   p.occ ? (float)p.occ[base] : 1.f);
        }
        __syncthreads();
        for (int i = 0; i < n; ++i) {
            const float4 a = stage[i];
            const T t0 = fma(Q0[0], (T)a.x, fma(Q0[1], (T)a.y, Q0[2] * (T)a.z));
            const T ts = fma(St[0], (T)a.x, fma(St[1], (T)a.y, St[2] * (T)a.z));
            T zr, zi, wr, wi2;
            sincos_cycles(frac_w(t0), zr, zi);
            sincos_cycles(frac_w(ts), wr, wi2);
            zr *= (T)a.w;
            zi *= (T)a.w;
#pragma unroll
            for (int j = 0; j < VPT; ++j) {
                acc[j] += zr;
                const T nr = fma(zr, wr, -zi * wi2);
                zi = fma(zr, wi2, zi * wr);
                zr = nr;
            }
        }
    }
    if (!live) return;
    const T inv = T(1) / (T)nsamp;
    const size_t v0 = ((size_t)i0 * p.cnt[1] + i1) * p.cnt[2] + i2_0;
#pragma unroll
    for (int j = 0; j < VPT; ++j)
        if (i2_0 + j < p.cnt[2]) p.out[(size_t)s * p.site_stride + v0 + j] = acc[j] * inv;
}

template <typename T> DwParams<T> dw_params(const ds_model *M, bool weights) {
    DwParams<T> d;
    memset(&d, 0, sizeof(d));
    d.nsite = M->nsite;
    d.ncell = M->n[0] * M->n[1] * M->n[2];
    d.nmodels = M->nmodels;
    d.disp = M->d_disp;
    d.occ = (weights && M->has_occ) ? M->d_occ : nullptr;
    for (int i = 0; i < 9; ++i) {
        d.recip[i] = M->recip[i];
        d.qstep[i] = M->recip[i] / M->n[i / 3];
    }
    return d;
}

template <typename T> void launch_dw(const DwParams<T> &d, cudaStream_t st) {
    const dim3 grid((unsigned)((d.npts + DW_THREADS - 1) / DW_THREADS), (unsigned)d.nsite);
    k_debye_waller<T><<<grid, DW_THREADS, 0, st>>>(d);
    count_launches(1);
}

template <typename T>
ds_status run_subbox_points(ds_model *Mdl, const std::vector<int4> &org, const double *hkl, long long npts,
                            int hkl_dev, const ds_opts *o, void *out, int out_dev, cudaStream_t st,
                            ds_result_info *info) {
    ds_ctx *ctx = Mdl->ctx;
    const int nsite = Mdl->nsite;
    const int kind = o->disorder == DS_OCC ? SB_OCC : (o->disorder == DS_SPIN ? SB_SPIN : SB_DISP);
    std::vector<SbSite> sites(nsite);
    for (int s = 0; s < nsite; ++s) {
        SbSite &S = sites[s];
        memset(&S, 0, sizeof(S));
        for (int a = 0; a < 3; ++a) S.r[a] = Mdl->sites[3 * s + a];
        S.b = Mdl->scat[s];
        S.kind = Mdl->ffkind[s];
        for (int j = 0; j < 9; ++j) S.coef[j] = Mdl->ffcoef[9 * s + j];
    }
    const long long norigin = (long long)org.size();
    const long long pblocks = (npts + SB_THREADS - 1) / SB_THREADS;
    const SbKernel<T> kern = subbox_kernel<T>(kind, nsite, kind == SB_DISP && Mdl->has_occ);
    int per_sm = 0, nsm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, SB_THREADS, 0) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ctx->device) != cudaSuccess)
        return ds_fail(ctx, DS_ERR_CUDA, "occupancy query failed");
    const long long per = origin_chunks(norigin, pblocks, (long long)std::max(1, per_sm) * std::max(1, nsm));
    const long long nchunk = (norigin + per - 1) / per;

    if (Mdl->ready) cudaStreamWaitEvent(st, Mdl->ready, 0);  // uploads made on another stream
    Scratch ws(st);
    SbSite *d_sites = (SbSite *)ws.get(sizeof(SbSite) * nsite);
    int4 *d_org = (int4 *)ws.get(sizeof(int4) * norigin);
    const double *d_hkl = hkl;
    if (!hkl_dev) d_hkl = (const double *)ws.get(sizeof(double) * 3 * npts);
    T *partial = (T *)ws.get(sizeof(T) * nchunk * npts);
    T *dw = (kind == SB_DISP && o->mode == DS_DIFFUSE) ? (T *)ws.get(sizeof(T) * nsite * npts) : nullptr;
    T *dout = out_dev ? (T *)out : (T *)ws.get(sizeof(T) * npts);
    if (ws.failed) return ds_fail(ctx, DS_ERR_OOM, "device allocation failed (sub-box points)");
    if (ws.total > ctx->budget)
        return ds_fail(ctx, DS_ERR_ADMISSION, "request needs %zu bytes of scratch, budget %zu", ws.total, ctx->budget);
    if (cudaMemcpyAsync(d_sites, sites.data(), sizeof(SbSite) * nsite, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(d_org, org.data(), sizeof(int4) * norigin, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        (!hkl_dev && cudaMemcpyAsync((void *)d_hkl, hkl, sizeof(double) * 3 * npts, cudaMemcpyHostToDevice, st) != cudaSuccess))
        return ds_fail(ctx, DS_ERR_CUDA, "copy of the sub-box inputs failed");
    if (dw) {
        ProfScope ps(ctx, "debye_waller", st);
        DwParams<T> d = dw_params<T>(Mdl, true);
        d.hkl = d_hkl;
        d.npts = npts;
        d.site_stride = npts;
        d.pt_stride = 1;
        d.out = dw;
        launch_dw<T>(d, st);
    }
    SbParams<T> p;
    memset(&p, 0, sizeof(p));
    p.nsite = nsite;
    p.nsb = o->subbox_n;
    p.n1 = Mdl->n[0];
    p.n2 = Mdl->n[1];
    p.n3 = Mdl->n[2];
    p.ncell = p.n1 * p.n2 * p.n3;
    p.diffuse = o->mode == DS_DIFFUSE;
    p.site = d_sites;
    p.occ = Mdl->has_occ ? Mdl->d_occ : nullptr;
    p.vec = kind == SB_SPIN ? Mdl->d_spins : Mdl->d_disp;
    p.mean = kind == SB_OCC ? (Mdl->user_mean ? Mdl->d_user_mean : Mdl->d_mean_occ) : Mdl->d_mean_spin;
    p.dw = dw;
    p.hkl = d_hkl;
    p.npts = npts;
    p.origins = d_org;
    p.norigin = norigin;
    p.per_chunk = per;
    for (int i = 0; i < 9; ++i) p.recip[i] = Mdl->recip[i];
    p.partial = partial;
    {
        ProfScope ps(ctx, "subbox_dft", st);
        kern<<<dim3((unsigned)pblocks, (unsigned)nchunk), SB_THREADS, 0, st>>>(p);
        double norm = 1.0 / ((double)norigin * nsite * (double)p.nsb * p.nsb * p.nsb);
        if (kind == SB_SPIN) norm *= 0.07265;  // C of Eq. mag_intensity (barn)
        const unsigned nb = (unsigned)std::max<long long>(1, std::min<long long>((npts + 255) / 256, 152 * 8));
        k_sum_chunks<T><<<nb, 256, 0, st>>>(partial, npts, (int)nchunk, norm, dout);
        count_launches(2);
    }
    if (cudaGetLastError() != cudaSuccess) return ds_fail(ctx, DS_ERR_CUDA, "sub-box launch failed");
    if (!out_dev && cudaMemcpyAsync(out, dout, sizeof(T) * npts, cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return ds_fail(ctx, DS_ERR_CUDA, "copy of the intensities to the host failed");
    ws.release();
    // the host tables above must outlive their queued copies
    if (cudaStreamSynchronize(st) != cudaSuccess)
        return ds_fail(ctx, DS_ERR_CUDA, "stream synchronisation failed: %s", cudaGetErrorString(cudaGetLastError()));
    if (info) {
        info->nvox = npts;
        info->workspace_bytes = (int64_t)ws.total;
    }
    return DS_OK;
}

template <typename T>
ds_status run_debye_waller(ds_model *Mdl, const double *hkl, long long npts, int hkl_dev, int weights, void *out,
                           int out_dev, cudaStream_t st) {
    ds_ctx *ctx = Mdl->ctx;
    if (Mdl->ready) cudaStreamWaitEvent(st, Mdl->ready, 0);
    Scratch ws(st);
    const double *d_hkl = hkl;
    if (!hkl_dev) d_hkl = (const double *)ws.get(sizeof(double) * 3 * npts);
    T *dout = out_dev ? (T *)out : (T *)ws.get(sizeof(T) * npts * Mdl->nsite);
    if (ws.failed) return ds_fail(ctx, DS_ERR_OOM, "device allocation failed (Debye-Waller)");
    if (!hkl_dev && cudaMemcpyAsync((void *)d_hkl, hkl, sizeof(double) * 3 * npts, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return ds_fail(ctx, DS_ERR_CUDA, "copy of the points failed");
    {
        ProfScope ps(ctx, "debye_waller", st);
        DwParams<T> d = dw_params<T>(Mdl, weights != 0);
        d.hkl = d_hkl;
        d.npts = npts;
        d.site_stride = 1;
        d.pt_stride = Mdl->nsite;
        d.out = dout;
        launch_dw<T>(d, st);
    }
    if (cudaGetLastError() != cudaSuccess) return ds_fail(ctx, DS_ERR_CUDA, "Debye-Waller launch failed");
    if (!out_dev && cudaMemcpyAsync(out, dout, sizeof(T) * npts * Mdl->nsite, cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return ds_fail(ctx, DS_ERR_CUDA, "copy of the factors to the host failed");
    ws.release();
    if (cudaStreamSynchronize(st) != cudaSuccess)
        return ds_fail(ctx, DS_ERR_CUDA, "stream synchronisation failed: %s", cudaGetErrorString(cudaGetLastError()));
    return DS_OK;
}

}  // namespace

// T_mu(G) on the computing grid of a magnetic request, [site][voxel] (api.cu)
template <typename T> void debye_waller_grid(const ds_model *M, const int g0[3], const int cnt[3], T *out, cudaStream_t st) {
    DwParams<T> d = dw_params<T>(M, false);
    for (int a = 0; a < 3; ++a) {
        d.g0[a] = g0[a];
        d.cnt[a] = cnt[a];
    }
    d.npts = (long long)cnt[0] * cnt[1] * cnt[2];
    d.site_stride = d.npts;
    d.pt_stride = 1;
    d.out = out;
    constexpr int VPT = 8;
    const long long nwork = (long long)cnt[0] * cnt[1] * ((cnt[2] + VPT - 1) / VPT);
    const dim3 grid((unsigned)((nwork + DW_THREADS - 1) / DW_THREADS), (unsigned)d.nsite);
    k_debye_waller_rows<T, VPT><<<grid, DW_THREADS, 0, st>>>(d);
    count_launches(1);
}
template void debye_waller_grid<float>(const ds_model *, const int *, const int *, float *, cudaStream_t);
template void debye_waller_grid<double>(const ds_model *, const int *, const int *, double *, cudaStream_t);

extern "C" ds_status ds_request_subbox_points(ds_model *Mdl, const int32_t *origins, int64_t norigin, const double *hkl,
                                              int64_t npts, int hkl_is_device, const ds_opts *o, void *out,
                                              int out_is_device, void *stream, ds_result_info *info) {
    if (!Mdl) return DS_ERR_ARG;
    ds_ctx *ctx = Mdl->ctx;
    if (!o) return ds_fail(ctx, DS_ERR_ARG, "null options");
    if (npts < 0 || norigin < 0) return ds_fail(ctx, DS_ERR_ARG, "negative point or origin count");
    if (npts > 0 && (!hkl || !out)) return ds_fail(ctx, DS_ERR_ARG, "null points or output");
    if ((origins == nullptr) != (norigin == 0))
        return ds_fail(ctx, DS_ERR_ARG, "origins must be NULL with norigin = 0 (every lattice point) or a list of norigin rows");
    if (!Mdl->has_lattice || !Mdl->has_cells || Mdl->nsite < 1) return ds_fail(ctx, DS_ERR_STATE, "model incomplete");
    if (o->precision != DS_FP32 && o->precision != DS_FP64) return ds_fail(ctx, DS_ERR_ARG, "precision");
    if (o->mode != DS_TOTAL && o->mode != DS_DIFFUSE) return ds_fail(ctx, DS_ERR_ARG, "mode");
    if (o->disorder < 0 || o->disorder > 2) return ds_fail(ctx, DS_ERR_ARG, "disorder");
    if (o->disorder == DS_OCC && !Mdl->has_occ) return ds_fail(ctx, DS_ERR_STATE, "no occupancies uploaded");
    if (o->disorder == DS_SPIN && !Mdl->has_spins) return ds_fail(ctx, DS_ERR_STATE, "no spins uploaded");
    if (o->disorder == DS_DISP && !Mdl->has_disp) return ds_fail(ctx, DS_ERR_STATE, "no displacements uploaded");
    if (Mdl->nsite > 16) return ds_fail(ctx, DS_ERR_UNSUPPORTED, "sub-boxes by direct summation handle up to 16 sites");
    for (int a = 0; a < 3; ++a)
        if (o->subbox_n < 1 || o->subbox_n > Mdl->n[a])
            return ds_fail(ctx, DS_ERR_ARG, "subbox_n must satisfy 1 <= n_sb <= n_alpha");
    std::vector<int4> org;
    if (origins) {
        org.resize((size_t)norigin);
        for (long long i = 0; i < norigin; ++i) {
            const int32_t *r = origins + 4 * i;
            if (r[0] < 0 || r[0] >= Mdl->nmodels || r[1] < 0 || r[1] >= Mdl->n[0] || r[2] < 0 || r[2] >= Mdl->n[1] ||
                r[3] < 0 || r[3] >= Mdl->n[2])
                return ds_fail(ctx, DS_ERR_ARG, "origin %lld = (%d, %d, %d, %d) outside the supercells", i, r[0], r[1],
                               r[2], r[3]);
            org[(size_t)i] = make_int4(r[0], r[1], r[2], r[3]);
        }
    } else {
        org.reserve((size_t)Mdl->nmodels * Mdl->n[0] * Mdl->n[1] * Mdl->n[2]);
        for (int m = 0; m < Mdl->nmodels; ++m)
            for (int i = 0; i < Mdl->n[0]; ++i)
                for (int j = 0; j < Mdl->n[1]; ++j)
                    for (int l = 0; l < Mdl->n[2]; ++l) org.push_back(make_int4(m, i, j, l));
    }
    if (info) memset(info, 0, sizeof(*info));
    if (npts == 0) return DS_OK;
    if (!hkl_is_device)
        for (long long i = 0; i < 3 * npts; ++i)
            if (!std::isfinite(hkl[i])) return ds_fail(ctx, DS_ERR_ARG, "point %lld is not finite", i / 3);
    if (cudaSetDevice(ctx->device) != cudaSuccess) return ds_fail(ctx, DS_ERR_CUDA, "cudaSetDevice");
    cudaStream_t st = (cudaStream_t)stream;
    if (o->precision == DS_FP64)
        return run_subbox_points<double>(Mdl, org, hkl, npts, hkl_is_device, o, out, out_is_device, st, info);
    return run_subbox_points<float>(Mdl, org, hkl, npts, hkl_is_device, o, out, out_is_device, st, info);
}

extern "C" ds_status ds_debye_waller(ds_model *Mdl, const double *hkl, int64_t npts, int hkl_is_device, int precision,
                                     int occupancy_weights, void *out, int out_is_device, void *stream) {
    if (!Mdl) return DS_ERR_ARG;
    ds_ctx *ctx = Mdl->ctx;
    if (npts < 0) return ds_fail(ctx, DS_ERR_ARG, "negative point count");
    if (npts > 0 && (!hkl || !out)) return ds_fail(ctx, DS_ERR_ARG, "null points or output");
    if (precision != DS_FP32 && precision != DS_FP64) return ds_fail(ctx, DS_ERR_ARG, "precision");
    if (!Mdl->has_lattice || !Mdl->has_cells || Mdl->nsite < 1) return ds_fail(ctx, DS_ERR_STATE, "model incomplete");
    if (!Mdl->has_disp) return ds_fail(ctx, DS_ERR_STATE, "no displacements uploaded");
    if (npts == 0) return DS_OK;
    if (!hkl_is_device)
        for (long long i = 0; i < 3 * npts; ++i)
            if (!std::isfinite(hkl[i])) return ds_fail(ctx, DS_ERR_ARG, "point %lld is not finite", i / 3);
    if (cudaSetDevice(ctx->device) != cudaSuccess) return ds_fail(ctx, DS_ERR_CUDA, "cudaSetDevice");
    cudaStream_t st = (cudaStream_t)stream;
    if (precision == DS_FP64)
        return run_debye_waller<double>(Mdl, hkl, npts, hkl_is_device, occupancy_weights, out, out_is_device, st);
    return run_debye_waller<float>(Mdl, hkl, npts, hkl_is_device, occupancy_weights, out, out_is_device, st);
}
