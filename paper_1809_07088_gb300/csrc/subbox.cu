// Exact sub-box averaging (Section V A) for occupancy and spin disorder.
//
// Every lattice point o is the origin of a box of n_sb^3 cells with open boundaries.  Summing
// |F_o(G)|^2 over all origins regroups into pair correlations: with fields x_p (p = site, or
// site and Cartesian component for spins),
//     sum_o |F_o(G)|^2 = sum_{p,q} P_p(G) conj(P_q(G)) S_pq(k),
//     S_pq(k) = sum_Delta w(Delta) C_pq(Delta) exp(+i k.Delta),
//     C_pq(Delta) = sum_models sum_R x_p(R + Delta) x_q(R)   (periodic),
//     w(Delta) = prod_alpha (n_sb - |Delta_alpha|),  |Delta_alpha| < n_sb,
// where P_p(G) = b f(|G|) exp(iG.r_mu) and w counts the pairs of cells of one box separated by
// Delta -- the triangular cutoff the paper identifies as the reason sub-boxes reduce noise.
// The windowed correlations are real fields on the supercell grid (zero outside the window),
// transformed by the library's R2C FFT; a per-voxel kernel then contracts the pair spectra
// (with delta_ab - G^_a G^_b between spin components).  Valid for n_sb <= n_alpha / 2.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "api_internal.h"
#include "internal.h"

using namespace ds;

namespace {

// one thread per (pair, Delta in the window); the result is placed at Delta mod n
template <typename T>
__global__ void k_subbox_corr(Geometry g, int nmodels, int nfield, int npair, const int2 *pairs, const T *x, int nsb,
                              T *wc) {
    const int wlen = 2 * nsb - 1;
    const int nd = wlen * wlen * wlen;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)npair * nd) return;
    const int pr = (int)(idx / nd);
    const int d = (int)(idx - (long long)pr * nd);
    const int d1 = d / (wlen * wlen) - (nsb - 1);
    const int d2 = (d / wlen) % wlen - (nsb - 1);
    const int d3 = d % wlen - (nsb - 1);
    const int2 pq = pairs[pr];
    const int n1 = g.n[0], n2 = g.n[1], n3 = g.n[2];
    double acc = 0.0;
    for (int m = 0; m < nmodels; ++m) {
        const T *xp = x + ((size_t)m * nfield + pq.x) * g.ncell;
        const T *xq = x + ((size_t)m * nfield + pq.y) * g.ncell;
        for (int r1 = 0; r1 < n1; ++r1) {
            const int s1 = ((r1 + d1) % n1 + n1) % n1;
            for (int r2 = 0; r2 < n2; ++r2) {
                const int s2 = ((r2 + d2) % n2 + n2) % n2;
                const T *rowq = xq + ((size_t)r1 * n2 + r2) * n3;
                const T *rowp = xp + ((size_t)s1 * n2 + s2) * n3;
                int s3 = ((d3 % n3) + n3) % n3;
                T part = T(0);
                for (int r3 = 0; r3 < n3; ++r3) {
                    part = fma(rowp[s3], rowq[r3], part);
                    if (++s3 == n3) s3 = 0;
                }
                acc += (double)part;
            }
        }
    }
    const double w = (double)(nsb - abs(d1)) * (nsb - abs(d2)) * (nsb - abs(d3));
    const int c1 = ((d1 % n1) + n1) % n1, c2 = ((d2 % n2) + n2) % n2, c3 = ((d3 % n3) + n3) % n3;
    wc[(size_t)pr * g.ncell + ((size_t)c1 * n2 + c2) * n3 + c3] = (T)(w * acc);
}

// fields x_p of the request: occupancy b(delta - c) or b delta; spins b(M - <M>) or b M
template <typename T>
__global__ void k_subbox_fields(int kind, int nmodels, int nsite, int ncell, int diffuse, const uint8_t *occ,
                                const float *spins, const double *mean, const double *scat, T *x) {
    const int nc = kind == SRC_SPIN ? 3 : 1;
    const size_t tot = (size_t)nmodels * nsite * nc * ncell;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < tot; i += (size_t)gridDim.x * blockDim.x) {
        const size_t cell = i % ncell;
        const size_t f = i / ncell;              // (m, site, comp)
        const int comp = (int)(f % nc);
        const int site = (int)((f / nc) % nsite);
        const int m = (int)(f / ((size_t)nc * nsite));
        double v;
        if (kind == SRC_SPIN) {
            v = spins[(((size_t)m * nsite + site) * ncell + cell) * 3 + comp];
            if (diffuse) v -= mean[site * 3 + comp];
        } else {
            v = occ[((size_t)m * nsite + site) * ncell + cell];
            if (diffuse) v -= mean[site];
        }
        x[i] = (T)(v * scat[site]);
    }
}

// per voxel: sum over pairs p <= q of (2 - delta_pq) Re[P_p conj(P_q) S_pq(k) M_ab(G)]
template <typename T, int NC, int MAXS>
__global__ void __launch_bounds__(256) k_subbox_recomb(const __grid_constant__ RecombParams<T> p, int npair,
                                                       const int2 *pairs, const c_t<T> *S) {
    using C = c_t<T>;
    const Geometry &g = p.g;
    const GridMap &gm = p.gm;
    const long long nv = (long long)gm.cnt[0] * gm.cnt[1] * gm.cnt[2];
    const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nv) return;
    const int i3 = (int)(v % gm.cnt[2]);
    const int i2 = (int)((v / gm.cnt[2]) % gm.cnt[1]);
    const int i1 = (int)(v / ((long long)gm.cnt[2] * gm.cnt[1]));
    const int G[3] = {gm.g0[0] + i1, gm.g0[1] + i2, gm.g0[2] + i3};
    int k[3], h[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        k[a] = ((G[a] % g.n[a]) + g.n[a]) % g.n[a];
        h[a] = (G[a] - k[a]) / g.n[a] - gm.Hmin[a];
    }
    double Qd[3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
        Qd[a] = (double)G[0] / g.n[0] * p.recip[a] + (double)G[1] / g.n[1] * p.recip[3 + a] +
                (double)G[2] / g.n[2] * p.recip[6 + a];
    const T q2 = (T)(Qd[0] * Qd[0] + Qd[1] * Qd[1] + Qd[2] * Qd[2]);
    const T s2 = q2 * (T)(1.0 / (FOUR_PI_D * FOUR_PI_D));
    T qh[3] = {T(0), T(0), T(0)};
    if (q2 > T(0)) {
        const T iq = T(1) / sqrt(q2);
#pragma unroll
        for (int a = 0; a < 3; ++a) qh[a] = (T)Qd[a] * iq;
    }
    // P_mu = f_mu(|G|) exp(iG.r_mu) (b is in the fields)
    C P[MAXS];
    int cls = 0;
    T f = form_factor<T>(p.ff.cls_kind[0], p.ff.cls_coef[0], s2);
#pragma unroll
    for (int s = 0; s < MAXS; ++s) {
        if (s < p.nsite) {
            if (s == p.ff.cls_end[cls]) {
                ++cls;
                f = form_factor<T>(p.ff.cls_kind[cls], p.ff.cls_coef[cls], s2);
            }
            const int site = p.site_of[s];
            const C *tH = p.phH + (size_t)site * 3 * p.nHmax;
            const C *tk = p.phk + (size_t)site * 3 * p.nmax;
            C ph = cmul(cmul(tH[h[0]], tH[p.nHmax + h[1]]), tH[2 * p.nHmax + h[2]]);
            ph = cmul(ph, cmul(cmul(tk[k[0]], tk[p.nmax + k[1]]), tk[2 * p.nmax + k[2]]));
            P[site < MAXS ? site : 0] = cscale(ph, f);
        }
    }
    int conj;
    const int kidx = half_index(g, k[0], k[1], k[2], conj);
    T acc = T(0);
    for (int pr = 0; pr < npair; ++pr) {
        const int2 pq = pairs[pr];
        const int mu = pq.x / NC, nu = pq.y / NC;
        C sv = S[(size_t)pr * g.ncell_h + kidx];
        if (conj) sv = cconj(sv);
        C pp = P[0], qq = P[0];
#pragma unroll
        for (int s = 0; s < MAXS; ++s) {
            if (s == mu) pp = P[s];
            if (s == nu) qq = P[s];
        }
        T wgt = (pq.x == pq.y) ? T(1) : T(2);
        if (NC == 3) {
            const int a = pq.x % 3, b = pq.y % 3;
            wgt *= (q2 > T(0)) ? ((a == b ? T(1) : T(0)) - qh[a] * qh[b]) : ((a == b) ? T(2) / T(3) : T(0));
        }
        const C t = cmul(cmulc(pp, qq), sv);
        acc = fma(wgt, t.x, acc);
    }
    p.out[v] = p.norm * acc;
}

// Residue-class contraction (sites on special positions, one form-factor class): with
// P_mu = f exp(iH.r_mu) exp(ik.r_mu), the pair sum of a voxel is
//     f^2 sum_{p<=q} (2 - delta_pq) Re[exp(iH.(r_mu - r_nu)) D_pq(k)] proj_ab(Q),
//     D_pq(k) = exp(ik.(r_mu - r_nu)) S_pq(k),
// and exp(iH.(r_mu - r_nu)) depends on H only through its residue class (see recomb_res.cu).  A
// thread owns one k and a class (rho1, rho2); it forms the class sums C_ab once per rho3 (for
// spins six sums, the off-diagonal ones holding both orders of a, b) and each voxel then costs
// f^2 (tr C - Q.C.Q / |Q|^2).
template <typename T, int NC, int D3>
__global__ void __launch_bounds__(128, 4)
    k_subbox_res(const __grid_constant__ RecombParams<T> p, const c_t<T> *S, int s3) {
    using C = c_t<T>;
    constexpr int NSYM = NC == 3 ? 6 : 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nsite = p.nsite, nf = nsite * NC;
    const int n1 = p.g.n[0], n2 = p.g.n[1], n3 = p.g.n[2];
    const int d1 = p.dres[0], d2 = p.dres[1], d3 = p.dres[2];
    const int part = blockIdx.y % s3;
    const int r12 = blockIdx.y / s3;
    const int rho1 = r12 / d2, rho2 = r12 - rho1 * d2;
    C *P123 = (C *)smem_raw;                                  // [d3][nsite]
    C *ek = P123 + (size_t)d3 * nsite;                        // [nsite][128]: exp(ik.r_mu)
    for (int idx = threadIdx.x; idx < d3 * nsite; idx += blockDim.x) {
        const int r3 = idx / nsite, s = idx - r3 * nsite;
        const C *t = p.phH + (size_t)s * 3 * p.nHmax;        // sites in input order
        P123[idx] = cmul(cmul(t[rho1], t[p.nHmax + rho2]), t[2 * p.nHmax + r3]);
    }
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const bool kvalid = k < p.g.ncell;
    const int kq = kvalid ? k : 0;
    const int k3 = kq % n3, k2 = (kq / n3) % n2, k1 = kq / (n3 * n2);
    for (int s = 0; s < nsite; ++s) {
        const C *t = p.phk + (size_t)s * 3 * p.nmax;
        ek[(size_t)s * blockDim.x + threadIdx.x] = cmul(cmul(t[k1], t[p.nmax + k2]), t[2 * p.nmax + k3]);
    }
    __syncthreads();
    if (!kvalid) return;
    int conj;
    const int kidx = half_index(p.g, k1, k2, k3, conj);
    const GridMap &gm = p.gm;
    const int g01 = gm.g0[0], g02 = gm.g0[1], g03 = gm.g0[2], cnt1 = gm.cnt[0], cnt2 = gm.cnt[1], cnt3 = gm.cnt[2];
    const int G1b = n1 * gm.Hmin[0] + k1, G2b = n2 * gm.Hmin[1] + k2, G3b = n3 * gm.Hmin[2] + k3;
    // zones h3 whose voxel G3 = G3b + n3 h3 lies in [g03, g03 + cnt3)
    auto fdiv = [](int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); };
    const int lo3 = max(-fdiv(-(g03 - G3b), n3), 0);
    const int h3hi = min(fdiv(g03 + cnt3 - 1 - G3b, n3), gm.nH[2] - 1);
    T qs[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) qs[i] = p.qstep[i];
    const T norm = p.norm;
    const int stride = n3 * d3;
    const int nchunk = (d3 + D3 - 1) / D3;
    const int lo3_mod = lo3 % d3;

    for (int ch = part; ch < nchunk; ch += s3) {
        const int r0 = ch * D3;
        T acc[D3][NSYM];
#pragma unroll
        for (int r = 0; r < D3; ++r)
#pragma unroll
            for (int c = 0; c < NSYM; ++c) acc[r][c] = T(0);
        for (int mu = 0; mu < nsite; ++mu) {
            const C emu = ek[(size_t)mu * blockDim.x + threadIdx.x];
            for (int nu = mu; nu < nsite; ++nu) {
                const C ekk = cmulc(emu, ek[(size_t)nu * blockDim.x + threadIdx.x]);  // e^{ik.(r_mu - r_nu)}
                C E[D3];
#pragma unroll
                for (int r = 0; r < D3; ++r)
                    E[r] = (r0 + r < d3) ? cmulc(P123[(size_t)(r0 + r) * nsite + mu], P123[(size_t)(r0 + r) * nsite + nu])
                                         : mk<T>(T(0), T(0));
#pragma unroll
                for (int a = 0; a < NC; ++a) {
#pragma unroll
                    for (int b = 0; b < NC; ++b) {
                        if (mu == nu && b < a) continue;
                        const int pf = mu * NC + a, qf = nu * NC + b;
                        const int pr = pf * nf - pf * (pf - 1) / 2 + (qf - pf);
                        C sv = S[(size_t)pr * p.g.ncell_h + kidx];
                        if (conj) sv = cconj(sv);
                        const T w = (pf == qf) ? T(1) : T(2);
                        const C D = cscale(cmul(ekk, sv), w);
                        const int c = NC == 3 ? (a <= b ? (a == 0 ? b : (a == 1 ? 2 + b : 5)) : (b == 0 ? a : (b == 1 ? 2 + a : 5))) : 0;
#pragma unroll
                        for (int r = 0; r < D3; ++r) acc[r][c] += E[r].x * D.x - E[r].y * D.y;
                    }
                }
            }
        }
#pragma unroll
        for (int r = 0; r < D3; ++r) {
            const int rho3 = r0 + r;
            if (rho3 >= d3) break;
            int t3 = rho3 - lo3_mod;
            if (t3 < 0) t3 += d3;
            const int h3s = lo3 + t3;
            if (h3s > h3hi) continue;
            const int nv3 = (h3hi - h3s) / d3 + 1;
            const int G3s = G3b + n3 * h3s;
            // class sums over component pairs (00, 01 + 10, 02 + 20, 11, 12 + 21, 22) times the norm
            T cm[NSYM];
#pragma unroll
            for (int c = 0; c < NSYM; ++c) cm[c] = acc[r][c] * norm;
            const T tr = NC == 3 ? cm[0] + cm[3] + cm[5] : cm[0];
            for (int h1 = rho1; h1 < gm.nH[0]; h1 += d1) {
                const int G1 = G1b + n1 * h1;
                if (G1 < g01 || G1 >= g01 + cnt1) continue;
                for (int h2 = rho2; h2 < gm.nH[1]; h2 += d2) {
                    const int G2 = G2b + n2 * h2;
                    if (G2 < g02 || G2 >= g02 + cnt2) continue;
                    T *row = p.out + ((size_t)(G1 - g01) * cnt2 + (G2 - g02)) * cnt3 + (G3s - g03);
                    T Qs[3];
#pragma unroll
                    for (int a = 0; a < 3; ++a) Qs[a] = fma((T)G3s, qs[6 + a], fma((T)G1, qs[a], (T)G2 * qs[3 + a]));
                    for (int i3 = 0; i3 < nv3; ++i3) {
                        T Qv[3];
#pragma unroll
                        for (int a = 0; a < 3; ++a) Qv[a] = fma((T)(i3 * stride), qs[6 + a], Qs[a]);
                        const T q2 = Qv[0] * Qv[0] + Qv[1] * Qv[1] + Qv[2] * Qv[2];
                        T val = tr;
                        if (NC == 3) {
                            // the off-diagonal sums already hold both orders (a, b) and (b, a)
                            const T qcq = cm[0] * Qv[0] * Qv[0] + cm[3] * Qv[1] * Qv[1] + cm[5] * Qv[2] * Qv[2] +
                                          cm[1] * Qv[0] * Qv[1] + cm[2] * Qv[0] * Qv[2] + cm[4] * Qv[1] * Qv[2];
                            val = q2 > T(0) ? tr - div_w(qcq, q2) : T(2) / T(3) * tr;
                        }
                        if (p.ff.cls_kind[0] != 0) {
                            const T f = form_factor<T>(p.ff.cls_kind[0], p.ff.cls_coef[0], q2 * (T)(1.0 / (FOUR_PI_D * FOUR_PI_D)));
                            val *= f * f;
                        }
                        row[(size_t)i3 * stride] = val;
                    }
                }
            }
        }
    }
}

}  // namespace

template <typename T>
ds_status subbox_run(ds_model *M, const ds_qgrid *q, const ds_opts *o, T *d_out, cudaStream_t st, Scratch &ws,
                     ds_result_info *info) {
    using C = c_t<T>;
    ds_ctx *ctx = M->ctx;
    int g0[3], cnt[3];
    ds_status rc = grid_indices(ctx, M, q, g0, cnt);
    if (rc != DS_OK) return rc;
    if (M->nsite > 16) return ds_fail(ctx, DS_ERR_UNSUPPORTED, "sub-box averaging handles up to 16 sites");
    if (!M->ff_ok) return ds_fail(ctx, DS_ERR_UNSUPPORTED, "too many distinct form factors");
    Geometry g;
    make_geometry(M->n, g);
    const GridMap gm = grid_map(g, g0, cnt);
    const int nsite = M->nsite, nmod = M->nmodels, nsb = o->subbox_n;
    const int kind = o->disorder == DS_SPIN ? SRC_SPIN : SRC_OCC;
    const int NC = kind == SRC_SPIN ? 3 : 1;
    const int nfield = nsite * NC;
    std::vector<int2> pairs;
    for (int a = 0; a < nfield; ++a)
        for (int b = a; b < nfield; ++b) pairs.push_back(make_int2(a, b));
    const int npair = (int)pairs.size();

    T *x = (T *)ws.get(sizeof(T) * (size_t)nmod * nfield * g.ncell);
    T *wc = (T *)ws.get(sizeof(T) * (size_t)npair * g.ncell);
    C *S = (C *)ws.get(sizeof(C) * (size_t)npair * g.ncell_h);
    const int fb = std::max(1, std::min(npair, (int)((256ull << 20) / (sizeof(C) * (size_t)g.ncell_h))));
    C *work = (C *)ws.get(sizeof(C) * (size_t)fb * g.ncell_h);
    int2 *d_pairs = (int2 *)ws.get(sizeof(int2) * npair);
    double *d_mean = (double *)ws.get(sizeof(double) * nsite * 3);
    double *d_scat = (double *)ws.get(sizeof(double) * nsite);
    RecombParams<T> p;
    memset(&p, 0, sizeof(p));
    p.nmax = std::max(g.n[0], std::max(g.n[1], g.n[2]));
    p.nHmax = std::max(gm.nH[0], std::max(gm.nH[1], gm.nH[2]));
    C *phk = (C *)ws.get(sizeof(C) * nsite * 3 * p.nmax);
    C *phH = (C *)ws.get(sizeof(C) * nsite * 3 * p.nHmax);
    if (ws.failed) return ds_fail(ctx, DS_ERR_OOM, "device allocation failed (sub-box buffers)");
    if (ws.total > ctx->budget)
        return ds_fail(ctx, DS_ERR_ADMISSION, "sub-box request needs %zu bytes of scratch, budget %zu", ws.total,
                       ctx->budget);
    if (M->ready) cudaStreamWaitEvent(st, M->ready, 0);  // uploads made on another stream
    cudaMemcpyAsync(d_pairs, pairs.data(), sizeof(int2) * npair, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(d_scat, M->scat.data(), sizeof(double) * nsite, cudaMemcpyHostToDevice, st);
    const bool diffuse = o->mode == DS_DIFFUSE;
    if (diffuse) {
        if (kind == SRC_SPIN) site_means_spin(nmod, nsite, g.ncell, M->d_spins, d_mean, st);
        else if (M->user_mean) cudaMemcpyAsync(d_mean, M->d_user_mean, sizeof(double) * nsite, cudaMemcpyDeviceToDevice, st);
        else site_means_occ(nmod, nsite, g.ncell, M->d_occ, d_mean, st);
    }
    {
        ProfScope ps(ctx, "subbox_corr", st);
        const size_t tot = (size_t)nmod * nfield * g.ncell;
        k_subbox_fields<T><<<(unsigned)std::min<size_t>((tot + 255) / 256, 152 * 32), 256, 0, st>>>(
            kind, nmod, nsite, g.ncell, diffuse, M->d_occ, M->d_spins, d_mean, d_scat, x);
        cudaMemsetAsync(wc, 0, sizeof(T) * (size_t)npair * g.ncell, st);
        const long long nd = (long long)npair * (2 * nsb - 1) * (2 * nsb - 1) * (2 * nsb - 1);
        k_subbox_corr<T><<<(unsigned)((nd + 127) / 128), 128, 0, st>>>(g, nmod, nfield, npair, d_pairs, x, nsb, wc);
        count_launches(2);
    }
    FieldSource src;
    memset(&src, 0, sizeof(src));
    src.kind = SRC_REAL;
    src.nf_per_model = npair;
    src.real_buf = wc;
    const C *W[3];
    for (int a = 0; a < 3; ++a) {
        if constexpr (sizeof(T) == 4) W[a] = M->d_tw32[a];
        else W[a] = M->d_tw64[a];
    }
    {
        ProfScope ps(ctx, "fft", st);
        for (int f0 = 0; f0 < npair; f0 += fb)
            fft_real_fields<T>(g, src, f0, std::min(fb, npair - f0), work, S, W[0], W[1], W[2], st);
    }
    make_site_tables<T>(g, gm, nsite, M->d_sites, phk, phH, p.nmax, p.nHmax, st);
    p.g = g;
    p.gm = gm;
    p.nsite = nsite;
    p.nmodels = nmod;
    p.phk = phk;
    p.phH = phH;
    p.nmax = std::max(g.n[0], std::max(g.n[1], g.n[2]));
    p.site_of = M->d_site_of;
    if constexpr (sizeof(T) == 4) p.ff = M->ff32;
    else p.ff = M->ff64;
    set_reciprocal(p, M->recip, g.n);
    double norm = 1.0 / ((double)nmod * g.ncell * nsite * (double)nsb * nsb * nsb);
    if (kind == SRC_SPIN) norm *= 0.07265;  // C of Eq. mag_intensity (barn)
    p.norm = (T)norm;
    p.out = d_out;
    const bool res = p.ff.ncls == 1 && residue_classes(M, gm, p.dres) &&
                     (size_t)p.dres[2] * nsite * sizeof(C) + (size_t)nsite * 128 * sizeof(C) <= 96 * 1024 &&
                     (long long)p.dres[0] * p.dres[1] * p.dres[2] <= 65535;
    if (res) {
        ProfScope ps(ctx, "subbox_recombine", st);
        constexpr int D3 = 4;
        const int ktiles = (g.ncell + 127) / 128;
        const int d12 = p.dres[0] * p.dres[1], nchunk = (p.dres[2] + D3 - 1) / D3;
        int s3 = nchunk;
        for (int c = 1; c <= nchunk; ++c)
            if (nchunk % c == 0 && (long long)ktiles * d12 * c >= 152LL * 4) { s3 = c; break; }
        const size_t sm = ((size_t)p.dres[2] * nsite + (size_t)nsite * 128) * sizeof(C);
        dim3 grid((unsigned)ktiles, (unsigned)(d12 * s3));
        if (NC == 1) {
            if (sm > 48 * 1024) cudaFuncSetAttribute(k_subbox_res<T, 1, D3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
            k_subbox_res<T, 1, D3><<<grid, 128, sm, st>>>(p, S, s3);
        } else {
            if (sm > 48 * 1024) cudaFuncSetAttribute(k_subbox_res<T, 3, D3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
            k_subbox_res<T, 3, D3><<<grid, 128, sm, st>>>(p, S, s3);
        }
        count_launches(1);
    } else {
        ProfScope ps(ctx, "subbox_recombine", st);
        const long long nv = (long long)cnt[0] * cnt[1] * cnt[2];
        const unsigned nb = (unsigned)((nv + 255) / 256);
        if (NC == 1) k_subbox_recomb<T, 1, 16><<<nb, 256, 0, st>>>(p, npair, d_pairs, S);
        else k_subbox_recomb<T, 3, 16><<<nb, 256, 0, st>>>(p, npair, d_pairs, S);
        count_launches(1);
    }
    if (cudaGetLastError() != cudaSuccess) return ds_fail(ctx, DS_ERR_CUDA, "sub-box launch failed");
    if (info) {
        info->taylor_order = 0;
        info->n_monomials = 0;
        info->x_max = -1.0;
        info->trunc_bound = 0.0;
    }
    return DS_OK;
}

template ds_status subbox_run<float>(ds_model *, const ds_qgrid *, const ds_opts *, float *, cudaStream_t, Scratch &,
                                     ds_result_info *);
template ds_status subbox_run<double>(ds_model *, const ds_qgrid *, const ds_opts *, double *, cudaStream_t,
                                      Scratch &, ds_result_info *);
