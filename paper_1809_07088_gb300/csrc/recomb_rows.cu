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
// Work split.  A CTA owns one (k1, k2) and one class rho1 of zone columns: every output row
// (G1, G2) with G1 = k1 (mod n1), G2 = k2 (mod n2), all G3.  It first forms the table of
// F(rho2, rho3, k3) over the d2 d3 n3 triples (per-site transforms of its (k1, k2) staged in
// shared memory, the site sum done once per entry), then writes its rows whole: thread t owns the
// voxels l = t + 64 j of every row, so the table entry, the axis-3 part of Q and the axis-3
// Gaussian factors of a voxel are per-thread constants reused over the rows, and each warp stores
// 128 consecutive bytes.  When the reciprocal axes are the Cartesian ones (cubic, tetragonal,
// orthorhombic cells) the form factor's Gaussians factor as exp(b (Qx^2 + Qy^2)) exp(b Qz^2), the
// first per row, the second per thread, so a voxel costs no transcendental (one reciprocal in the
// magnetic case).  In FP32 the table sums and the per-voxel arithmetic run on pairs (FFMA2).
//
// Friedel pairs.  The densities are real, so F(-G) = conj F(G) and I(-G) = I(G) for both
// intensities (Q -> -Q leaves |Q.F|^2 unchanged).  -G = n (-H - [k != 0]) + (-k mod n) lies in the
// rows of the CTA of (-k1, -k2) and the class of -H1 - [k1 != 0]; of each such pair of CTAs the
// lower-numbered one computes its voxels and writes every one also at -G when -G is in the grid,
// and the other computes only the voxels whose -G lies outside the grid (none when the grid is
// symmetric about the origin, in which case it returns at once).  A CTA paired with itself
// computes all of its voxels.  Every voxel is written by exactly one thread.
#include <algorithm>
#include <climits>
#include <cmath>

#include "internal.h"

namespace ds {

namespace {

constexpr int RW_THREADS = 128;
constexpr int RW_GROUP = 64;    // threads writing one row
constexpr int RW_SLOTS = 4;     // voxels of a row per thread per pass (pairs for FFMA2)
constexpr int RW_ROWS = 64;     // row constants staged per pass
constexpr int RW_MAXNG = 4;
constexpr int RW_RB = 3;        // table entries per thread per pass (register blocking)
constexpr long long RW_NOMIRROR = LLONG_MIN;

// floor division and non-negative remainder by a launch constant 1 <= d <= 2^14, for |x| < 2^16, as a
// multiply-high by m = ceil(2^32 / d) = (2^32 + e) / d, 0 <= e < d: with u = x + K d (K d > 2^16, so
// 0 < u < 2^17 + d) and u = q d + r, umulhi(u, m) = q + floor((r + u e / 2^32) / d) = q because
// u e < u d < 2^32.  d = 1 has m = 0 and takes u itself.
struct SDiv {
    int d, K, Kd;
    unsigned m;
    void set(int dd) {
        d = dd;
        K = (1 << 16) / dd + 1;
        Kd = K * dd;
        m = FastDiv::magic((unsigned)dd);
    }
    __device__ __forceinline__ int div(int x) const {
        const unsigned u = (unsigned)(x + Kd);
        return (int)(m ? __umulhi(u, m) : u) - K;
    }
    __device__ __forceinline__ int mod(int x) const { return x - d * div(x); }
};

// launch constants of the row kernel (host-computed)
struct RowsAux {
    SDiv n1, n2, n3, d1, d2, d3, d23;
    int rs;            // RW_THREADS / n3: threads per k3 in the staging and the table
    int dq, dk, dqm;   // RW_GROUP = dq n3 + dk, dqm = dq mod d3: step between a thread's slots
    int symm;          // the grid is symmetric about the origin on every axis
};

// pairs of the working type: packed FP32 (FFMA2 / FMUL2 / FADD2) or two FP64 operations
template <typename T> struct Pair;
template <> struct Pair<float> {
    using t = float2;
};
template <> struct Pair<double> {
    using t = double2;
};
__device__ __forceinline__ float2 pfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 pmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 padd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ double2 pfma(double2 a, double2 b, double2 c) {
    return make_double2(fma(a.x, b.x, c.x), fma(a.y, b.y, c.y));
}
__device__ __forceinline__ double2 pmul(double2 a, double2 b) { return make_double2(a.x * b.x, a.y * b.y); }
__device__ __forceinline__ double2 padd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
template <typename T> __device__ __forceinline__ typename Pair<T>::t pmk(T a, T b) { return {a, b}; }

// shared-memory layout (byte offsets, 16-byte aligned).  PW: per site and class (rho2, rho3) the
// phase w as (w.x, w.x, -w.y, w.y) in FP32 (the two FFMA2 multiplicands), w itself in FP64; YS: per
// site, component and k3 the weighted transform y (8 bytes in FP32: the swapped pair (y.y, y.x) the
// second FFMA2 needs is formed in registers, once per load and reused over the classes)
struct RowsLayout {
    size_t PW, YS, tab, rq, re, ro, mo, total;
};
__host__ __device__ __forceinline__ RowsLayout rows_layout(int nsite, int nc, int n3, int d2, int d3, size_t te) {
    auto al = [](size_t x) { return (x + 15) & ~(size_t)15; };
    const int tw = nc == 3 ? 8 : 1;
    RowsLayout L;
    L.PW = 0;
    L.YS = al(L.PW + (size_t)nsite * d2 * d3 * 16);
    L.tab = al(L.YS + (size_t)nsite * nc * n3 * 2 * te);
    L.rq = al(L.tab + (size_t)d2 * d3 * n3 * tw * te);
    L.re = al(L.rq + (size_t)2 * RW_ROWS * 4 * te);
    L.ro = al(L.re + (size_t)2 * RW_ROWS * RW_MAXNG * te);
    L.mo = al(L.ro + (size_t)2 * RW_ROWS * sizeof(long long));
    L.total = al(L.mo + (size_t)2 * RW_ROWS * sizeof(long long));
    return L;
}

// acc += w y for complex w, y: FP32 from the packed forms (two FFMA2), FP64 directly
__device__ __forceinline__ void tab_fma(float2 &acc, const float4 &w, const float2 &y) {
    acc = __ffma2_rn(make_float2(w.x, w.y), y, acc);
    acc = __ffma2_rn(make_float2(w.z, w.w), make_float2(y.y, y.x), acc);
}
__device__ __forceinline__ void tab_fma(double2 &acc, const double2 &w, const double2 &y) {
    acc.x = fma(w.x, y.x, fma(-w.y, y.y, acc.x));
    acc.y = fma(w.x, y.y, fma(w.y, y.x, acc.y));
}
template <typename T> struct Packed;
template <> struct Packed<float> {
    using t = float4;
    static __device__ __forceinline__ float4 phase(float2 w) { return make_float4(w.x, w.x, -w.y, w.y); }
    using y = float2;
    static __device__ __forceinline__ float2 value(float2 v) { return v; }
};
template <> struct Packed<double> {
    using t = double2;
    static __device__ __forceinline__ double2 phase(double2 w) { return w; }
    using y = double2;
    static __device__ __forceinline__ double2 value(double2 v) { return v; }
};

}  // namespace

// NC: 1 (occupancy) or 3 (moments); NG: Gaussians of the form factor (0 = constant); ORTHO: the
// reciprocal axes are the Cartesian ones; ACC: add into the output (later supercells of the ensemble)
template <typename T, int NC, int NG, bool ORTHO, bool ACC>
__global__ void __launch_bounds__(RW_THREADS, sizeof(T) == 4 ? 6 : 3)
    k_recomb_rows(const __grid_constant__ RecombParams<T> p, const RowsAux ax) {
    using C = c_t<T>;
    using V = typename Pair<T>::t;
    using PK = Packed<T>;
    using PT = typename PK::t;
    constexpr int TW = NC == 3 ? 8 : 1;
    extern __shared__ __align__(16) unsigned char smem[];
    const int n1 = p.g.n[0], n2 = p.g.n[1], n3 = p.g.n[2];
    const int d1 = p.dres[0], d2 = p.dres[1], d3 = p.dres[2];
    const int blk = blockIdx.x;
    const int b12 = ax.n2.div(blk), k2 = blk - b12 * n2;
    const int rho1 = ax.n1.div(b12), k1 = b12 - rho1 * n1;
    const GridMap &gm = p.gm;

    // Friedel partner CTA and this CTA's role: 0 alone, 1 writes its voxels and their mirrors,
    // 2 writes only the voxels whose mirror lies outside the grid
    const int k1m = k1 ? n1 - k1 : 0, k2m = k2 ? n2 - k2 : 0;
    const int rho1m = ax.d1.mod(-2 * gm.Hmin[0] - rho1 - (k1 != 0));
    const int bm = (rho1m * n1 + k1m) * n2 + k2m;
    const int role = bm == blk ? 0 : (blk < bm ? 1 : 2);
    const bool symm = ax.symm != 0;
    if (role == 2 && symm) return;

    // zones of the grid along axes 1 and 2 for this k; axis 1 restricted to the CTA's class rho1
    const int h1lo = max(-ax.n1.div(k1 - gm.g0[0]) - gm.Hmin[0], 0);
    const int h1hi = min(ax.n1.div(gm.g0[0] + gm.cnt[0] - 1 - k1) - gm.Hmin[0], gm.nH[0] - 1);
    const int h2lo = max(-ax.n2.div(k2 - gm.g0[1]) - gm.Hmin[1], 0);
    const int h2hi = min(ax.n2.div(gm.g0[1] + gm.cnt[1] - 1 - k2) - gm.Hmin[1], gm.nH[1] - 1);
    const int f1 = h1lo + ax.d1.mod(rho1 - h1lo);
    const int nr1 = f1 <= h1hi ? ax.d1.div(h1hi - f1) + 1 : 0;
    const int nh2 = h2hi >= h2lo ? h2hi - h2lo + 1 : 0;
    if (nr1 * nh2 == 0) return;

    const int nsite = p.nsite, d23 = d2 * d3;
    const RowsLayout L = rows_layout(nsite, NC, n3, d2, d3, sizeof(T));
    PT *PW = (PT *)(smem + L.PW);
    using YT = typename PK::y;
    YT *YS = (YT *)(smem + L.YS);
    T *tab = (T *)(smem + L.tab);
    T *rq = (T *)(smem + L.rq);
    T *re = (T *)(smem + L.re);
    long long *ro = (long long *)(smem + L.ro);
    long long *mo = (long long *)(smem + L.mo);
    const int tid = threadIdx.x;
    const int nmax = p.nmax, nHmax = p.nHmax;
    const size_t nh = p.g.ncell_h;
    // each thread keeps one k3 for the staging and the table: rows rr, rr + rs, ... of the site and
    // class lists (n3 <= 128)
    const int rr = ax.n3.div(tid), q3 = tid - rr * n3, rs = ax.rs;
    const bool tb = rr < rs;

    // zone phases of the classes (rho1, rho2, rho3) per site.  With one form-factor class the site
    // sum takes every site once in any order: sites by their own index, no sorted-order lookup.
    // (the loads of RW_SB entries or sites are issued together, then combined: the staging is
    // bound by the latency of these loads)
    constexpr int RW_SB = 4;
    for (int i0 = tid; i0 < nsite * d23; i0 += RW_SB * RW_THREADS) {
        C h[RW_SB][3];
#pragma unroll
        for (int u = 0; u < RW_SB; ++u) {
            const int i = i0 + u * RW_THREADS;
            if (i < nsite * d23) {
                const int s = ax.d23.div(i), r23 = i - s * d23, r2 = ax.d3.div(r23), r3 = r23 - r2 * d3;
                const C *tH = p.phH + (size_t)s * 3 * nHmax;
                h[u][0] = __ldg(tH + rho1);
                h[u][1] = __ldg(tH + nHmax + r2);
                h[u][2] = __ldg(tH + 2 * nHmax + r3);
            }
        }
#pragma unroll
        for (int u = 0; u < RW_SB; ++u) {
            const int i = i0 + u * RW_THREADS;
            if (i < nsite * d23) PW[i] = PK::phase(cmul(h[u][0], cmul(h[u][1], h[u][2])));
        }
    }
    // everything below reads the spectra (and the output): the transform that wrote them, when it
    // ran just before this kernel, must have completed
    griddep_wait();
    // y_mu,c(k) = b exp(ik.r_mu) X_mu,c(k) of the thread's k3, every component
    if (tb) {
        // stored half k3 < n3h; the other half from -k with conj (0 <= k_a < n_a)
        const int conj = q3 >= p.g.n3h;
        const int kidx = conj ? (k1m * n2 + k2m) * p.g.n3h + (n3 - q3) : (k1 * n2 + k2) * p.g.n3h + q3;
        const C *spec = p.spec + (size_t)p.model * nsite * NC * nh + kidx;
        for (int sp0 = rr; sp0 < nsite; sp0 += RW_SB * rs) {
            C t[RW_SB][3], x[RW_SB][NC];
            T b[RW_SB];
#pragma unroll
            for (int u = 0; u < RW_SB; ++u) {
                const int sp = sp0 + u * rs;
                if (sp < nsite) {
                    const C *tk = p.phk + (size_t)sp * 3 * nmax;
                    t[u][0] = __ldg(tk + k1);
                    t[u][1] = __ldg(tk + nmax + k2);
                    t[u][2] = __ldg(tk + 2 * nmax + q3);
                    b[u] = __ldg(p.scat + sp);
#pragma unroll
                    for (int c = 0; c < NC; ++c) x[u][c] = __ldg(spec + (size_t)(sp * NC + c) * nh);
                }
            }
#pragma unroll
            for (int u = 0; u < RW_SB; ++u) {
                const int sp = sp0 + u * rs;
                if (sp < nsite) {
                    const C w = cscale(cmul(cmul(t[u][0], t[u][1]), t[u][2]), b[u]);
#pragma unroll
                    for (int c = 0; c < NC; ++c)
                        YS[(sp * NC + c) * n3 + q3] = PK::value(cmul(w, conj ? cconj(x[u][c]) : x[u][c]));
                }
            }
        }
    }
    __syncthreads();
    // table F(rho2, rho3, k3) = sum_mu exp(iH.r_mu) y_mu(k) (scaled by sqrt(norm)), norm |F|^2;
    // RW_RB classes per thread per pass share the loads of y
    const T sn = sqrt(p.norm);
    if (tb)
        for (int r0 = rr; r0 < d23; r0 += rs * RW_RB) {
            V F[RW_RB][NC];
            int rc[RW_RB];
#pragma unroll
            for (int i = 0; i < RW_RB; ++i) {
                rc[i] = min(r0 + rs * i, d23 - 1);
#pragma unroll
                for (int c = 0; c < NC; ++c) F[i][c] = pmk<T>(T(0), T(0));
            }
            for (int sp = 0; sp < nsite; ++sp) {
                YT y[NC];
#pragma unroll
                for (int c = 0; c < NC; ++c) y[c] = YS[(sp * NC + c) * n3 + q3];
#pragma unroll
                for (int i = 0; i < RW_RB; ++i) {
                    const PT w = PW[sp * d23 + rc[i]];
#pragma unroll
                    for (int c = 0; c < NC; ++c) tab_fma(F[i][c], w, y[c]);
                }
            }
#pragma unroll
            for (int i = 0; i < RW_RB; ++i) {
                const int r23 = r0 + rs * i;
                if (r23 >= d23) break;
                T tot = T(0);
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    F[i][c].x *= sn;
                    F[i][c].y *= sn;
                    tot = fma(F[i][c].x, F[i][c].x, fma(F[i][c].y, F[i][c].y, tot));
                }
                T *t = tab + (size_t)(r23 * n3 + q3) * TW;
                if (NC == 3) {
#pragma unroll
                    for (int c = 0; c < 3; ++c) t[2 * c] = F[i][c].x, t[2 * c + 1] = F[i][c].y;
                    t[6] = tot;
                    t[7] = T(0);
                } else {
                    t[0] = tot;
                }
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
    // per pass along axis 3); the rows of a chunk alternate between the groups
    const int grp = tid / RW_GROUP, lt = tid - grp * RW_GROUP;
    const int dk = ax.dk, dqm = ax.dqm;

    // Rows in chunks: the rows (i1, h2) of one axis-2 class rho2 (h2 = rho2 mod d2), RW_ROWS at a
    // time; the constants of the next chunk are staged while the current one is written, in
    // alternating buffers, so one barrier per chunk suffices.
    // first non-empty class >= r2 (d2 if none), its first zone index h2 and its number of h2
    auto next_class = [&](int r2, int &fh2, int &nc2) {
        for (; r2 < d2; ++r2) {
            fh2 = h2lo + ax.d2.mod(r2 - h2lo);
            if (fh2 <= h2hi) {
                nc2 = ax.d2.div(h2hi - fh2) + 1;
                return r2;
            }
        }
        return d2;
    };
    // row constants of a chunk: output offsets (the row and its mirror), Q of the row (axes 1, 2),
    // Gaussian factors of axes 1, 2
    auto stage = [&](int buf, int c0, int fh2, int nc2) {
        const int nr = min(RW_ROWS, nr1 * nc2 - c0), b0 = buf * RW_ROWS;
        for (int r = tid; r < nr; r += RW_THREADS) {
            const int i1 = (c0 + r) / nc2, h2 = fh2 + d2 * ((c0 + r) - i1 * nc2);
            const int G1 = n1 * (gm.Hmin[0] + f1 + d1 * i1) + k1, G2 = n2 * (gm.Hmin[1] + h2) + k2;
            ro[b0 + r] = ((long long)(G1 - gm.g0[0]) * gm.cnt[1] + (G2 - gm.g0[1])) * cnt3;
            const int M1 = -G1 - gm.g0[0], M2 = -G2 - gm.g0[1];
            const bool mir = role != 0 && M1 >= 0 && M1 < gm.cnt[0] && M2 >= 0 && M2 < gm.cnt[1];
            mo[b0 + r] = mir ? ((long long)M1 * gm.cnt[1] + M2) * cnt3 - 2LL * g03 : RW_NOMIRROR;
            T Q[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) Q[a] = fma((T)G1, qs[a], (T)G2 * qs[3 + a]);
            const T q12 = ORTHO ? fma(Q[0], Q[0], Q[1] * Q[1]) : T(0);
            T *q = rq + 4 * (b0 + r);
            q[0] = Q[0];
            q[1] = Q[1];
            q[2] = Q[2];
            q[3] = q12;
#pragma unroll
            for (int g = 0; g < RW_MAXNG; ++g)
                re[RW_MAXNG * (b0 + r) + g] = (ORTHO && g < NG) ? ga[g] * exp2_w(gb[g] * q12) : T(0);
        }
    };
    int fh2_0 = 0, nc2_0 = 0;
    const int r2_0 = next_class(0, fh2_0, nc2_0);
    if (r2_0 < d2) stage(0, 0, fh2_0, nc2_0);
    __syncthreads();   // the table and the first chunk's row constants are complete

    for (int l0 = 0; l0 < cnt3; l0 += RW_GROUP * RW_SLOTS) {
        // per-slot constants: table column, axis-3 part of Q and of the Gaussians, and whether the
        // voxel and its mirror -G3 lie in the grid
        int ev[RW_SLOTS];
        bool vz[RW_SLOTS], mz[RW_SLOTS];
        T q3v[RW_SLOTS][ORTHO ? 1 : 3];   // orthogonal axes: Qz only
        V nqz2[RW_SLOTS / 2], e3[RW_SLOTS / 2][RW_MAXNG];
        {
            const int G3 = g03 + l0 + lt;
            const int zq = ax.n3.div(G3);
            int kk = G3 - zq * n3, hr = ax.d3.mod(zq - gm.Hmin[2]);
#pragma unroll
            for (int j = 0; j < RW_SLOTS; ++j) {
                const int l = l0 + lt + RW_GROUP * j, G3j = g03 + l;
                ev[j] = hr * n3 + kk;
                vz[j] = l < cnt3;
                mz[j] = -G3j >= g03 && -G3j < g03 + cnt3;
                if (ORTHO) {
                    q3v[j][0] = (T)G3j * qs[8];
                } else {
#pragma unroll
                    for (int a = 0; a < (ORTHO ? 1 : 3); ++a) q3v[j][a] = (T)G3j * qs[6 + a];
                }
                // next slot: G3 + RW_GROUP
                kk += dk;
                int carry = 0;
                if (kk >= n3) kk -= n3, carry = 1;
                hr += dqm + carry;
                if (hr >= d3) hr -= d3;
                if (hr >= d3) hr -= d3;
            }
#pragma unroll
            for (int j = 0; j < RW_SLOTS; j += 2) {
                const T qz0 = q3v[j][ORTHO ? 0 : 2], qz1 = q3v[j + 1][ORTHO ? 0 : 2];
                const T z0 = qz0 * qz0, z1 = qz1 * qz1;
                nqz2[j / 2] = pmk<T>(-z0, -z1);
#pragma unroll
                for (int g = 0; g < RW_MAXNG; ++g)
                    e3[j / 2][g] = (ORTHO && g < NG) ? pmk<T>(exp2_w(gb[g] * z0), exp2_w(gb[g] * z1)) : pmk<T>(T(0), T(0));
            }
        }
        if (l0 > 0) {
            // a further pass along axis 3: the first chunk again
            if (r2_0 < d2) stage(0, 0, fh2_0, nc2_0);
            __syncthreads();
        }
        // the current class's table entries of the slots, as pairs; the axis-3 part of Q.F
        // (orthogonal axes) or F2 itself
        V tot[RW_SLOTS / 2], F0r[RW_SLOTS / 2], F0i[RW_SLOTS / 2], F1r[RW_SLOTS / 2], F1i[RW_SLOTS / 2],
            czr[RW_SLOTS / 2], czi[RW_SLOTS / 2];
        int loaded = -1;
        int cr2 = r2_0, cfh2 = fh2_0, cnc2 = nc2_0, cc0 = 0;
        for (int it = 0; cr2 < d2; ++it) {
            // stage the next chunk
            int nr2 = cr2, nfh2 = cfh2, nnc2 = cnc2, nc0 = cc0 + RW_ROWS;
            if (nc0 >= nr1 * cnc2) {
                nr2 = next_class(cr2 + 1, nfh2, nnc2);
                nc0 = 0;
            }
            if (nr2 < d2) stage((it + 1) & 1, nc0, nfh2, nnc2);
            if (cr2 != loaded) {
                loaded = cr2;
#pragma unroll
                for (int h = 0; h < RW_SLOTS / 2; ++h) {
                    T e[2][8];
#pragma unroll
                    for (int u = 0; u < 2; ++u) {
                        const int j = 2 * h + u;
                        const T *t = tab + ((size_t)cr2 * d3 * n3 + ev[j]) * TW;
                        if (NC == 3) {
                            if (sizeof(T) == 4) {
                                const float4 a = ((const float4 *)t)[0], c = ((const float4 *)t)[1];
                                e[u][0] = a.x, e[u][1] = a.y, e[u][2] = a.z, e[u][3] = a.w;
                                e[u][4] = c.x, e[u][5] = c.y, e[u][6] = c.z;
                            } else {
#pragma unroll
                                for (int q = 0; q < 7; ++q) e[u][q] = t[q];
                            }
                            const T s3 = ORTHO ? q3v[j][0] : T(1);
                            e[u][4] *= s3;
                            e[u][5] *= s3;
                        } else {
                            e[u][6] = t[0];
                        }
                    }
                    tot[h] = pmk<T>(e[0][6], e[1][6]);
                    if (NC == 3) {
                        F0r[h] = pmk<T>(e[0][0], e[1][0]);
                        F0i[h] = pmk<T>(e[0][1], e[1][1]);
                        F1r[h] = pmk<T>(e[0][2], e[1][2]);
                        F1i[h] = pmk<T>(e[0][3], e[1][3]);
                        czr[h] = pmk<T>(e[0][4], e[1][4]);
                        czi[h] = pmk<T>(e[0][5], e[1][5]);
                    }
                }
            }
            const int nr = min(RW_ROWS, nr1 * cnc2 - cc0), b0 = (it & 1) * RW_ROWS;
            for (int r = b0 + grp; r < b0 + nr; r += RW_THREADS / RW_GROUP) {
                const long long mrow = mo[r];
                const bool hasm = mrow != RW_NOMIRROR;
                T *row = out + ro[r] + l0 + lt;
                T *mrw = hasm ? out + (mrow - l0 - lt) : out;
                const T Qx = rq[4 * r], Qy = rq[4 * r + 1], Qz0 = rq[4 * r + 2], q12 = rq[4 * r + 3];
                T val[RW_SLOTS];
                if (ORTHO && (NC == 1 || q12 > T(0))) {
                    // paired evaluation (no voxel of the row has Q = 0)
                    const V Qx2 = pmk<T>(Qx, Qx), Qy2 = pmk<T>(Qy, Qy), nq12 = pmk<T>(-q12, -q12);
                    V er2[RW_MAXNG];
#pragma unroll
                    for (int g = 0; g < RW_MAXNG; ++g) {
                        const T e = g < NG ? re[RW_MAXNG * r + g] : T(0);
                        er2[g] = pmk<T>(e, e);
                    }
#pragma unroll
                    for (int h = 0; h < RW_SLOTS / 2; ++h) {
                        V v = tot[h];
                        if (NC == 3) {
                            const V pr = pfma(Qx2, F0r[h], pfma(Qy2, F1r[h], czr[h]));
                            const V pi = pfma(Qx2, F0i[h], pfma(Qy2, F1i[h], czi[h]));
                            const V pp = pfma(pr, pr, pmul(pi, pi));
                            const V nq2 = padd(nq12, nqz2[h]);           // -|Q|^2
                            v = pfma(pp, pmk<T>(rcp_w(nq2.x), rcp_w(nq2.y)), v);
                        }
                        if (NG > 0) {
                            V f = pmk<T>(gc, gc);
#pragma unroll
                            for (int g = 0; g < NG; ++g) f = pfma(er2[g], e3[h][g], f);
                            v = pmul(v, pmul(f, f));
                        }
                        val[2 * h] = v.x;
                        val[2 * h + 1] = v.y;
                    }
                } else {
#pragma unroll
                    for (int h = 0; h < RW_SLOTS / 2; ++h)
#pragma unroll
                        for (int u = 0; u < 2; ++u) {
                            const int j = 2 * h + u;
                            // orthogonal axes: |Q|^2 = q12 + Qz^2 from the stored -Qz^2
                            const T Qv0 = ORTHO ? Qx : Qx + q3v[j][ORTHO ? 0 : 0];
                            const T Qv1 = ORTHO ? Qy : Qy + q3v[j][ORTHO ? 0 : 1];
                            const T Qv2 = ORTHO ? Qz0 : Qz0 + q3v[j][ORTHO ? 0 : 2];
                            const T q2 = ORTHO ? q12 - (u ? nqz2[h].y : nqz2[h].x) : fma(Qv0, Qv0, fma(Qv1, Qv1, Qv2 * Qv2));
                            const T tt = u ? tot[h].y : tot[h].x;
                            T v = tt;
                            if (NC == 3) {
                                const T a0 = u ? F0r[h].y : F0r[h].x, b0v = u ? F0i[h].y : F0i[h].x;
                                const T a1 = u ? F1r[h].y : F1r[h].x, b1 = u ? F1i[h].y : F1i[h].x;
                                const T a2 = u ? czr[h].y : czr[h].x, b2 = u ? czi[h].y : czi[h].x;
                                // orthogonal axes: a2, b2 hold Qz F2; otherwise F2
                                const T pr = ORTHO ? fma(Qx, a0, fma(Qy, a1, a2)) : fma(Qv0, a0, fma(Qv1, a1, Qv2 * a2));
                                const T pi = ORTHO ? fma(Qx, b0v, fma(Qy, b1, b2)) : fma(Qv0, b0v, fma(Qv1, b1, Qv2 * b2));
                                const T pp = fma(pr, pr, pi * pi);
                                v = q2 > T(0) ? fma(-pp, rcp_w(q2), tt) : T(2) / T(3) * tt;
                            }
                            if (NG > 0) {
                                T f = gc;
#pragma unroll
                                for (int g = 0; g < NG; ++g) {
                                    const T e3g = u ? e3[h][g].y : e3[h][g].x;
                                    f = ORTHO ? fma(re[RW_MAXNG * r + g], e3g, f) : fma(ga[g], exp2_w(gb[g] * q2), f);
                                }
                                v *= f * f;
                            }
                            val[j] = v;
                        }
                }
                if (symm && role == 1) {
                    // symmetric grid: every voxel of the row has its mirror in the grid
#pragma unroll
                    for (int j = 0; j < RW_SLOTS; ++j) {
                        if (!vz[j]) continue;
                        T *dst = row + RW_GROUP * j, *mdst = mrw - RW_GROUP * j;
                        if (ACC) *dst += val[j], *mdst += val[j];
                        else *dst = val[j], *mdst = val[j];
                    }
                    continue;
                }
#pragma unroll
                for (int j = 0; j < RW_SLOTS; ++j) {
                    const bool mw = hasm && mz[j];
                    // the partner of a mirrored pair skips what its partner writes
                    if (!vz[j] || (role == 2 && mw)) continue;
                    T *dst = row + RW_GROUP * j;
                    if (ACC) *dst += val[j];
                    else *dst = val[j];
                    if (role == 1 && mw) {
                        T *mdst = mrw - RW_GROUP * j;
                        if (ACC) *mdst += val[j];
                        else *mdst = val[j];
                    }
                }
            }
            __syncthreads();   // the chunk's buffer is free; the next chunk's constants are staged
            cr2 = nr2, cfh2 = nfh2, cnc2 = nnc2, cc0 = nc0;
        }
    }
}

template <typename T, int NC, int NG, bool ORTHO, bool ACC> static void launch_rows(const RecombParams<T> &p, cudaStream_t s) {
    const RowsLayout L = rows_layout(p.nsite, NC, p.g.n[2], p.dres[1], p.dres[2], sizeof(T));
    const unsigned nblk = (unsigned)p.g.n[0] * p.g.n[1] * p.dres[0];
    RowsAux ax;
    ax.n1.set(p.g.n[0]);
    ax.n2.set(p.g.n[1]);
    ax.n3.set(p.g.n[2]);
    ax.d1.set(p.dres[0]);
    ax.d2.set(p.dres[1]);
    ax.d3.set(p.dres[2]);
    ax.d23.set(p.dres[1] * p.dres[2]);
    ax.rs = RW_THREADS / p.g.n[2];
    ax.dq = RW_GROUP / p.g.n[2];
    ax.dk = RW_GROUP - ax.dq * p.g.n[2];
    ax.dqm = ax.dq % p.dres[2];
    ax.symm = 1;
    for (int a = 0; a < 3; ++a) ax.symm &= 2 * p.gm.g0[a] + p.gm.cnt[a] == 1;
    if (L.total > 48 * 1024)
        cudaFuncSetAttribute(k_recomb_rows<T, NC, NG, ORTHO, ACC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.total);
    // programmatic dependent launch: the CTAs may start (decoding, zone phases) while the
    // transform before them in the stream finishes; they wait for it before reading its output
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nblk);
    cfg.blockDim = dim3(RW_THREADS);
    cfg.dynamicSmemBytes = L.total;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, k_recomb_rows<T, NC, NG, ORTHO, ACC>, p, ax);
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
// transforms within 96 KB of shared memory
template <typename T> bool recombine_rows(const RecombParams<T> &p, cudaStream_t s) {
    if (p.dres[0] <= 0 || p.ff.ncls != 1 || p.force_plain || p.Fout || p.dw) return false;
    if (p.ff.cls_ng[0] > RW_MAXNG) return false;
    // the multiply-high divisions: divisors up to 2^14, coordinates below 2^16 in magnitude
    if (p.g.n[0] > RW_THREADS || p.g.n[1] > RW_THREADS || p.g.n[2] > RW_THREADS) return false;
    if ((long long)p.dres[1] * p.dres[2] > (1 << 14) || p.dres[0] > (1 << 14)) return false;
    for (int a = 0; a < 3; ++a)
        if (std::abs(p.gm.g0[a]) + (long long)p.gm.cnt[a] + 2LL * std::abs(p.gm.Hmin[a]) + 2LL * p.g.n[a] >= (1 << 15))
            return false;
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
