// Row-wise recombination for sites on special positions with one form-factor class
// (compositional and magnetic; Section III B, Eq. comp_sf_diffuse, and Section III D, Eqs. mag_sf,
// mag_intensity, mag_projection).
//
// With G = H + k (Eq. g_vec) and every site coordinate along axis a a multiple of 1/d_a, the zone
// phase exp(2 pi i H_a r_mu,a) depends on H_a only through H_a mod d_a (the residue class rho_a), so
//     F_c(G) = sum_mu exp(iH.r_mu) b_mu exp(ik.r_mu) X_mu,c(k)
// takes one value per (rho, k).  With a single form factor f(|Q|) common to the sites, the
// intensity of voxel G is
//     I(G) = f^2 norm |F|^2                                    (occupancy)
//     I(G) = f^2 norm (|F|^2 - |Q.F|^2 / |Q|^2)                  (moments; (2/3)|F|^2 at Q = 0)
// with F = F(rho, k): the same sum as the per-voxel recombination with the zone phases taken at
// the class representative, identical up to rounding.
//
// Work split.  A CTA owns one (k1, k2) and one class (rho1, rho2) of zone columns: every output row
// (G1, G2) with G1 = k1 (mod n1), G2 = k2 (mod n2) in those classes, all G3.  It first forms the
// table of F(rho3, k3) over the d3 n3 pairs (per-site transforms of its (k1, k2) staged in shared
// memory, the site sum done once per entry), then writes its rows whole: thread t owns the voxels
// l = t + 128 j of every row, so the table entry, the axis-3 part of Q and the axis-3 Gaussian
// factors of a voxel are per-thread constants reused over the rows, and each warp stores 128
// consecutive bytes.  When the reciprocal axes are the Cartesian ones (cubic, tetragonal,
// orthorhombic cells) the form factor's Gaussians factor as exp(b (Qx^2 + Qy^2)) exp(b Qz^2),
// the first per row, the second per thread, so a voxel costs no transcendental (one reciprocal in
// the magnetic case).  Every voxel is written by exactly one thread.
#include <algorithm>
#include <cmath>

#include "internal.h"

namespace ds {

namespace {

constexpr int RW_THREADS = 128;
constexpr int RW_GROUP = 64;    // threads writing one row
constexpr int RW_SLOTS = 4;     // voxels of a row per thread per pass
constexpr int RW_ROWS = 64;     // row constants staged per pass
constexpr int RW_MAXNG = 4;

__device__ __forceinline__ int fl_div(int a, int b) {
    int q = a / b;
    if ((a % b != 0) && ((a < 0) != (b < 0))) --q;
    return q;
}
__device__ __forceinline__ int pos_mod(int a, int b) {
    const int r = a % b;
    return r < 0 ? r + b : r;
}

// shared-memory layout (byte offsets, 16-byte aligned)
struct RowsLayout {
    size_t A, P23, X, tab, rq, re, ro, total;
};
__host__ __device__ __forceinline__ RowsLayout rows_layout(int nsite, int nc, int n3, int d2, int d3, size_t te) {
    auto al = [](size_t x) { return (x + 15) & ~(size_t)15; };
    const size_t ce = 2 * te;
    const int tw = nc == 3 ? 8 : 1;
    RowsLayout L;
    L.A = 0;
    L.P23 = al(L.A + (size_t)nsite * ce);
    L.X = al(L.P23 + (size_t)nsite * d2 * d3 * ce);
    L.tab = al(L.X + (size_t)nsite * nc * n3 * ce);
    L.rq = al(L.tab + (size_t)d2 * d3 * n3 * tw * te);
    L.re = al(L.rq + (size_t)RW_ROWS * 4 * te);
    L.ro = al(L.re + (size_t)RW_ROWS * RW_MAXNG * te);
    L.total = al(L.ro + (size_t)RW_ROWS * sizeof(long long));
    return L;
}

}  // namespace

// NC: 1 (occupancy) or 3 (moments); NG: Gaussians of the form factor (0 = constant); ORTHO: the
// reciprocal axes are the Cartesian ones; ACC: add into the output (later supercells of the ensemble)
template <typename T, int NC, int NG, bool ORTHO, bool ACC>
__global__ void __launch_bounds__(RW_THREADS) k_recomb_rows(const __grid_constant__ RecombParams<T> p) {
    using C = c_t<T>;
    constexpr int TW = NC == 3 ? 8 : 1;
    extern __shared__ __align__(16) unsigned char smem[];
    const int n1 = p.g.n[0], n2 = p.g.n[1], n3 = p.g.n[2];
    const int d1 = p.dres[0], d2 = p.dres[1], d3 = p.dres[2];
    int b = blockIdx.x;
    const int k2 = b % n2;
    b /= n2;
    const int k1 = b % n1;
    const int rho1 = b / n1;
    const GridMap &gm = p.gm;
    // zones of the grid along axes 1 and 2 for this k; axis 1 restricted to the CTA's class rho1
    const int h1lo = max(-fl_div(-(gm.g0[0] - k1), n1) - gm.Hmin[0], 0);
    const int h1hi = min(fl_div(gm.g0[0] + gm.cnt[0] - 1 - k1, n1) - gm.Hmin[0], gm.nH[0] - 1);
    const int h2lo = max(-fl_div(-(gm.g0[1] - k2), n2) - gm.Hmin[1], 0);
    const int h2hi = min(fl_div(gm.g0[1] + gm.cnt[1] - 1 - k2, n2) - gm.Hmin[1], gm.nH[1] - 1);
    const int f1 = h1lo + pos_mod(rho1 - h1lo, d1);
    const int nr1 = f1 <= h1hi ? (h1hi - f1) / d1 + 1 : 0;
    const int nh2 = h2hi >= h2lo ? h2hi - h2lo + 1 : 0;
    const int nrows = nr1 * nh2;
    if (nrows == 0) return;

    const int nsite = p.nsite, d23 = d2 * d3;
    const RowsLayout L = rows_layout(nsite, NC, n3, d2, d3, sizeof(T));
    C *A = (C *)(smem + L.A);
    C *P23 = (C *)(smem + L.P23);
    C *Xs = (C *)(smem + L.X);
    T *tab = (T *)(smem + L.tab);
    T *rq = (T *)(smem + L.rq);
    T *re = (T *)(smem + L.re);
    long long *ro = (long long *)(smem + L.ro);
    const int tid = threadIdx.x;
    const int nmax = p.nmax, nHmax = p.nHmax;
    const size_t nh = p.g.ncell_h;
    // each thread keeps one k3 for the table build: rows rr, rr + rs, ... of the (site, component)
    // and class lists
    const int q3 = tid % n3, rr = tid / n3, rs = RW_THREADS / n3;
    const bool tb = rr < rs;

    // b exp(i(k1, k2).r) per site, and the zone phases of the classes (rho1, rho2, rho3)
    for (int s = tid; s < nsite; s += RW_THREADS) {
        const C *tk = p.phk + (size_t)p.site_of[s] * 3 * nmax;
        A[s] = cscale(cmul(tk[k1], tk[nmax + k2]), p.scat[p.site_of[s]]);
    }
    for (int i = tid; i < nsite * d23; i += RW_THREADS) {
        const int s = i / d23, r23 = i - s * d23, r2 = r23 / d3, r3 = r23 - r2 * d3;
        const C *tH = p.phH + (size_t)p.site_of[s] * 3 * nHmax;
        P23[i] = cmul(tH[rho1], cmul(tH[nHmax + r2], tH[2 * nHmax + r3]));
    }
    int conj = 0;
    const int kidx = half_index(p.g, k1, k2, q3, conj);
    const C *spec = p.spec + (size_t)p.model * nsite * NC * nh + kidx;
    if (tb)
        for (int sc = rr; sc < nsite * NC; sc += rs) {
            const int sp = sc / NC, c = sc - sp * NC;
            const C x = spec[(size_t)(p.site_of[sp] * NC + c) * nh];
            Xs[sc * n3 + q3] = conj ? cconj(x) : x;
        }
    __syncthreads();
    // Y_mu,c(k) = b exp(ik.r_mu) X_mu,c(k), in place
    if (tb)
        for (int sc = rr; sc < nsite * NC; sc += rs) {
            const int sp = sc / NC;
            const C w = cmul(A[sp], p.phk[((size_t)p.site_of[sp] * 3 + 2) * nmax + q3]);
            Xs[sc * n3 + q3] = cmul(w, Xs[sc * n3 + q3]);
        }
    __syncthreads();
    // table F(rho2, rho3, k3) = sum_mu exp(iH.r_mu) Y_mu(k) (scaled by sqrt(norm)), norm |F|^2
    const T sn = sqrt(p.norm);
    if (tb)
        for (int r23 = rr; r23 < d23; r23 += rs) {
            C F[NC];
#pragma unroll
            for (int c = 0; c < NC; ++c) F[c] = mk<T>(T(0), T(0));
            for (int sp = 0; sp < nsite; ++sp) {
                const C w = P23[sp * d23 + r23];
#pragma unroll
                for (int c = 0; c < NC; ++c) cfma(F[c], w, Xs[(sp * NC + c) * n3 + q3]);
            }
            T tot = T(0);
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                F[c] = cscale(F[c], sn);
                tot += F[c].x * F[c].x + F[c].y * F[c].y;
            }
            T *t = tab + (size_t)(r23 * n3 + q3) * TW;
            if (NC == 3) {
#pragma unroll
                for (int c = 0; c < 3; ++c) t[2 * c] = F[c].x, t[2 * c + 1] = F[c].y;
                t[6] = tot;
                t[7] = T(0);
            } else {
                t[0] = tot;
            }
        }

    // form-factor coefficients (Gaussian sums in |Q|^2)
    T ga[RW_MAXNG], gb[RW_MAXNG];
#pragma unroll
    for (int i = 0; i < RW_MAXNG; ++i) ga[i] = p.ff.cls_ga[0][i], gb[i] = p.ff.cls_gb[0][i];
    const T gc = p.ff.cls_gc[0];
    const T *qs = p.qstep;
    const int g03 = gm.g0[2], cnt3 = gm.cnt[2];
    T *const out = p.out;
    // two groups of RW_GROUP threads, each writing whole rows (RW_SLOTS voxels of a row per thread
    // per pass along axis 3); the rows of one class rho2 alternate between the groups
    const int grp = tid / RW_GROUP, lt = tid - grp * RW_GROUP;
    __syncthreads();   // the table is complete

    for (int l0 = 0; l0 < cnt3; l0 += RW_GROUP * RW_SLOTS) {
        // per-slot constants: table column, axis-3 part of Q and of the Gaussians
        int ev[RW_SLOTS], lv[RW_SLOTS];
        T q3v[RW_SLOTS][3], qz2[RW_SLOTS], e3[RW_SLOTS][RW_MAXNG];
#pragma unroll
        for (int j = 0; j < RW_SLOTS; ++j) {
            const int l = l0 + lt + RW_GROUP * j;
            lv[j] = l;
            const int G3 = g03 + min(l, cnt3 - 1);
            const int h3 = fl_div(G3, n3) - gm.Hmin[2];
            ev[j] = (h3 % d3) * n3 + pos_mod(G3, n3);
#pragma unroll
            for (int a = 0; a < 3; ++a) q3v[j][a] = (T)G3 * qs[6 + a];
            qz2[j] = q3v[j][2] * q3v[j][2];
#pragma unroll
            for (int g = 0; g < RW_MAXNG; ++g) e3[j][g] = (ORTHO && g < NG) ? exp2_w(gb[g] * qz2[j]) : T(0);
        }
        for (int r2 = 0; r2 < d2; ++r2) {
            const int fh2 = h2lo + pos_mod(r2 - h2lo, d2);   // first h2 of the class
            if (fh2 > h2hi) continue;
            const int nc2 = (h2hi - fh2) / d2 + 1, ncls = nr1 * nc2;
            // the class's table entries of the slots, and the axis-3 part of Q.F
            T tot[RW_SLOTS], F0[RW_SLOTS][2], F1[RW_SLOTS][2], cz[RW_SLOTS][2];
#pragma unroll
            for (int j = 0; j < RW_SLOTS; ++j) {
                const T *t = tab + ((size_t)r2 * d3 * n3 + ev[j]) * TW;
                if (NC == 3) {
                    T F2[2];
                    if (sizeof(T) == 4) {
                        const float4 u = ((const float4 *)t)[0], v = ((const float4 *)t)[1];
                        F0[j][0] = u.x, F0[j][1] = u.y, F1[j][0] = u.z, F1[j][1] = u.w, F2[0] = v.x, F2[1] = v.y;
                        tot[j] = v.z;
                    } else {
                        F0[j][0] = t[0], F0[j][1] = t[1], F1[j][0] = t[2], F1[j][1] = t[3], F2[0] = t[4], F2[1] = t[5];
                        tot[j] = t[6];
                    }
                    // orthogonal axes: the axis-3 part of Q.F; otherwise F2 itself
                    cz[j][0] = ORTHO ? q3v[j][2] * F2[0] : F2[0];
                    cz[j][1] = ORTHO ? q3v[j][2] * F2[1] : F2[1];
                } else {
                    tot[j] = t[0];
                }
            }
            for (int c0 = 0; c0 < ncls; c0 += RW_ROWS) {
                const int nr = min(RW_ROWS, ncls - c0);
                __syncthreads();
                // row constants: output offset, Q of the row (axes 1, 2), Gaussian factors of axes 1, 2
                for (int r = tid; r < nr; r += RW_THREADS) {
                    const int i1 = (c0 + r) / nc2, h2 = fh2 + d2 * ((c0 + r) - i1 * nc2);
                    const int G1 = n1 * (gm.Hmin[0] + f1 + d1 * i1) + k1, G2 = n2 * (gm.Hmin[1] + h2) + k2;
                    ro[r] = ((long long)(G1 - gm.g0[0]) * gm.cnt[1] + (G2 - gm.g0[1])) * cnt3;
                    T Q[3];
#pragma unroll
                    for (int a = 0; a < 3; ++a) Q[a] = fma((T)G1, qs[a], (T)G2 * qs[3 + a]);
                    const T q12 = ORTHO ? fma(Q[0], Q[0], Q[1] * Q[1]) : T(0);
                    rq[4 * r] = Q[0];
                    rq[4 * r + 1] = Q[1];
                    rq[4 * r + 2] = Q[2];
                    rq[4 * r + 3] = q12;
#pragma unroll
                    for (int g = 0; g < RW_MAXNG; ++g) re[RW_MAXNG * r + g] = (ORTHO && g < NG) ? ga[g] * exp2_w(gb[g] * q12) : T(0);
                }
                __syncthreads();
                for (int r = grp; r < nr; r += RW_THREADS / RW_GROUP) {
                    T *row = out + ro[r];
                    const T Qx = rq[4 * r], Qy = rq[4 * r + 1], Qz0 = rq[4 * r + 2], q12 = rq[4 * r + 3];
                    T er[RW_MAXNG];
#pragma unroll
                    for (int g = 0; g < RW_MAXNG; ++g) er[g] = (ORTHO && g < NG) ? re[RW_MAXNG * r + g] : T(0);
#pragma unroll
                    for (int j = 0; j < RW_SLOTS; ++j) {
                        if (lv[j] >= cnt3) continue;
                        T val, q2 = T(0);
                        if (ORTHO) {
                            q2 = q12 + qz2[j];
                            if (NC == 3) {
                                const T pr = fma(Qx, F0[j][0], fma(Qy, F1[j][0], cz[j][0]));
                                const T pi = fma(Qx, F0[j][1], fma(Qy, F1[j][1], cz[j][1]));
                                const T pp = fma(pr, pr, pi * pi);
                                val = q2 > T(0) ? fma(-pp, rcp_w(q2), tot[j]) : T(2) / T(3) * tot[j];
                            } else {
                                val = tot[j];
                            }
                        } else {
                            const T Qv0 = Qx + q3v[j][0], Qv1 = Qy + q3v[j][1], Qv2 = Qz0 + q3v[j][2];
                            q2 = fma(Qv0, Qv0, fma(Qv1, Qv1, Qv2 * Qv2));
                            if (NC == 3) {
                                const T pr = fma(Qv0, F0[j][0], fma(Qv1, F1[j][0], Qv2 * cz[j][0]));
                                const T pi = fma(Qv0, F0[j][1], fma(Qv1, F1[j][1], Qv2 * cz[j][1]));
                                const T pp = fma(pr, pr, pi * pi);
                                val = q2 > T(0) ? fma(-pp, rcp_w(q2), tot[j]) : T(2) / T(3) * tot[j];
                            } else {
                                val = tot[j];
                            }
                        }
                        if (NG > 0) {
                            T f = gc;
                            if (ORTHO) {
#pragma unroll
                                for (int g = 0; g < NG; ++g) f = fma(er[g], e3[j][g], f);
                            } else {
#pragma unroll
                                for (int g = 0; g < NG; ++g) f = fma(ga[g], exp2_w(gb[g] * q2), f);
                            }
                            val *= f * f;
                        }
                        T *dst = row + lv[j];
                        if (ACC) *dst += val;
                        else *dst = val;
                    }
                }
            }
        }
    }
}

template <typename T, int NC, int NG, bool ORTHO, bool ACC> static void launch_rows(const RecombParams<T> &p, cudaStream_t s) {
    const RowsLayout L = rows_layout(p.nsite, NC, p.g.n[2], p.dres[1], p.dres[2], sizeof(T));
    const unsigned nblk = (unsigned)p.g.n[0] * p.g.n[1] * p.dres[0];
    if (L.total > 48 * 1024)
        cudaFuncSetAttribute(k_recomb_rows<T, NC, NG, ORTHO, ACC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.total);
    k_recomb_rows<T, NC, NG, ORTHO, ACC><<<nblk, RW_THREADS, L.total, s>>>(p);
    count_launches(1);
}

template <typename T, int NC, int NG> static void launch_rows_o(const RecombParams<T> &p, bool ortho, cudaStream_t s) {
    if (ortho) {
        if (p.accumulate) launch_rows<T, NC, NG, true, true>(p, s);
        else launch_rows<T, NC, NG, true, false>(p, s);
    } else {
        if (p.accumulate) launch_rows<T, NC, NG, false, true>(p, s);
        else launch_rows<T, NC, NG, false, false>(p, s);
    }
}

template <typename T, int NC> static void launch_rows_ng(const RecombParams<T> &p, bool ortho, cudaStream_t s) {
    const int ng = p.ff.cls_kind[0] == 0 ? 0 : p.ff.cls_ng[0];
    if (ng == 0) launch_rows_o<T, NC, 0>(p, ortho, s);
    else if (ng <= 2) launch_rows_o<T, NC, 2>(p, ortho, s);
    else launch_rows_o<T, NC, 4>(p, ortho, s);
}

// the row kernel when it applies: residue classes, one form-factor class, the table and the staged
// transforms within 48 KB of shared memory
template <typename T> bool recombine_rows(const RecombParams<T> &p, cudaStream_t s) {
    if (p.dres[0] <= 0 || p.ff.ncls != 1 || p.force_plain || p.Fout || p.dw) return false;
    if (p.ff.cls_ng[0] > RW_MAXNG) return false;
    const int nc = p.ncomp;
    if (rows_layout(p.nsite, nc, p.g.n[2], p.dres[1], p.dres[2], sizeof(T)).total > 96 * 1024) return false;
    if ((long long)p.g.n[0] * p.g.n[1] * p.dres[0] >= (1LL << 31)) return false;
    // reciprocal axes along x, y, z (cubic, tetragonal, orthorhombic in the standard setting)
    double dmax = 0.0, off = 0.0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            const double v = fabs(p.recip[3 * i + j]);
            if (i == j) dmax = std::max(dmax, v);
            else off = std::max(off, v);
        }
    const bool ortho = off <= 1e-12 * dmax;
    if (nc == 3) launch_rows_ng<T, 3>(p, ortho, s);
    else launch_rows_ng<T, 1>(p, ortho, s);
    return true;
}

template bool recombine_rows<float>(const RecombParams<float> &, cudaStream_t);
template bool recombine_rows<double>(const RecombParams<double> &, cudaStream_t);

}  // namespace ds
