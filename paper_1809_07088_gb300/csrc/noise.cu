// Noise reduction (Section V).
//
// Lanczos resampling on the commensurate grid (Section V B): for Q on the supercell Bragg
// grid, Eq. (intensity_convol_finite) with W = W_sinc L (Eqs. weight_sinc, windowed_sinc,
// lanczos) separates into three one-axis passes, each a (2h+1)-tap stencil with weights
//     w(d) = sinc(2 pi r_cut d) sinc(pi d / m_eff),  |d| < m_eff,
// normalised to unit sum (the 8 r_cut^3 prefactor and the denominator of Eq.
// intensity_convol_finite both cancel in the normalisation).  r_cut = (1 - 1/m)/m' and
// m_eff = m m' / 2 (m' = 2 is the plain window; larger m' reaches zero at 1/m').  Each pass
// shrinks the volume by the halo h = ceil(m_eff) - 1 on both sides of its axis.  Stencils of up
// to 17 taps run as two streaming passes: the two in-plane axes fused (one read of the
// halo-extended volume, one write of the intermediate), then the strided outer axis as a sliding
// window (one read, one write): HBM bound, about 16 bytes per FP32 voxel.  Wider stencils take one
// thread per output and one pass per axis.
#include <algorithm>
#include <cstdint>
#include <type_traits>

#include "internal.h"
#include "noise.h"

namespace ds {

template <typename T>
__global__ void k_lanczos_axis(const T *__restrict__ in, T *__restrict__ out, int d0, int d1, int d2, int axis,
                               int h, double rcut, double meff) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *w = (T *)smem_raw;
    const int ntap = 2 * h + 1;
    if (threadIdx.x == 0) {
        double tmp[64];
        double sum = 0.0;
        for (int i = 0; i < ntap; ++i) {
            const double d = (double)(i - h);
            double v = 0.0;
            if (fabs(d) < meff) {
                const double x1 = 2.0 * rcut * d, x2 = d / meff;  // in units of pi
                const double s1 = (d == 0.0) ? 1.0 : sinpi(x1) / (3.141592653589793238462643383279502884 * x1);
                const double s2 = (d == 0.0) ? 1.0 : sinpi(x2) / (3.141592653589793238462643383279502884 * x2);
                v = s1 * s2;
            }
            tmp[i] = v;
            sum += v;
        }
        for (int i = 0; i < ntap; ++i) w[i] = (T)(tmp[i] / sum);
    }
    __syncthreads();
    // output dims
    const int o0 = d0 - (axis == 0 ? 2 * h : 0);
    const int o1 = d1 - (axis == 1 ? 2 * h : 0);
    const int o2 = d2 - (axis == 2 ? 2 * h : 0);
    const size_t total = (size_t)o0 * o1 * o2;
    const size_t stride = axis == 0 ? (size_t)d1 * d2 : (axis == 1 ? (size_t)d2 : 1);
    for (size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x; v < total; v += (size_t)gridDim.x * blockDim.x) {
        const int i2 = (int)(v % o2);
        const int i1 = (int)((v / o2) % o1);
        const int i0 = (int)(v / ((size_t)o2 * o1));
        const size_t src = ((size_t)i0 * d1 + i1) * d2 + i2;  // start of the tap window
        T acc = T(0);
        for (int t = 0; t < ntap; ++t) acc = fma(w[t], in[src + (size_t)t * stride], acc);
        out[v] = acc;
    }
}

int lanczos_halo(int m, int mprime) {
    const double meff = 0.5 * m * mprime;
    return (int)ceil(meff) - 1;
}

// normalised one-axis stencil of (2h+1) taps, FP64 on the host
static void lanczos_taps(int h, double rcut, double meff, double *w) {
    const double pi = 3.141592653589793238462643383279502884;
    double sum = 0.0;
    for (int i = 0; i <= 2 * h; ++i) {
        const double d = (double)(i - h);
        double v = 0.0;
        if (fabs(d) < meff) {
            v = 1.0;
            if (d != 0.0) {
                const double x1 = pi * 2.0 * rcut * d, x2 = pi * d / meff;
                v = (sin(x1) / x1) * (sin(x2) / x2);
            }
        }
        w[i] = v;
        sum += v;
    }
    for (int i = 0; i <= 2 * h; ++i) w[i] /= sum;
}

template <typename T> struct Taps {
    T w[64];
};

// Pass along the middle axis of a volume viewed as [A][B][C] (C contiguous): out[a][b][c] =
// sum_t w_t in[a][b + t][c], b < B - 2h.  A thread owns one (a, c) column and a run of L
// outputs along B, keeping the last NT inputs in registers (a sliding window), so each input is
// read about (L + NT - 1) / L times; consecutive threads take consecutive c (coalesced).  The
// inputs of LM_U outputs are loaded together, so that many loads are in flight per thread.
constexpr int LM_U = 8;
template <typename T, int NT>
__global__ void __launch_bounds__(256) k_lanczos_mid(const T *__restrict__ in, T *__restrict__ out, int A, int B, int C,
                                                     int L, const __grid_constant__ Taps<T> tp) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int Bo = B - (NT - 1);
    const int nrun = (Bo + L - 1) / L;
    const int a = blockIdx.y / nrun, run = blockIdx.y - a * nrun;
    if (c >= C || a >= A) return;
    const int b0 = run * L, b1 = min(Bo, b0 + L);
    const T *src = in + ((size_t)a * B + b0) * C + c;
    T *dst = out + ((size_t)a * Bo + b0) * C + c;
    T ring[NT];
#pragma unroll
    for (int t = 0; t < NT - 1; ++t) ring[t] = src[(size_t)t * C];
    for (int b = b0; b < b1; b += LM_U) {
        T nx[LM_U];
#pragma unroll
        for (int u = 0; u < LM_U; ++u) nx[u] = b + u < b1 ? src[(size_t)(b - b0 + u + NT - 1) * C] : T(0);
#pragma unroll
        for (int u = 0; u < LM_U; ++u) {
            ring[NT - 1] = nx[u];
            T acc = T(0);
#pragma unroll
            for (int t = 0; t < NT; ++t) acc = fma(tp.w[t], ring[t], acc);
            if (b + u < b1) dst[(size_t)(b - b0 + u) * C] = acc;
#pragma unroll
            for (int t = 0; t < NT - 1; ++t) ring[t] = ring[t + 1];
        }
    }
}

// Fused in-plane pass over [A][B][C] (C contiguous): out[a][b][c] = sum_s w_s sum_t w_t
// in[a][b + s][c + t] for b < B - 2h, c < C - 2h.  A CTA owns a segment of W = 2 x blockDim
// outputs along C and a run of L outputs along B of one a; it streams the run's L + NT - 1 input
// rows through a ring of D row buffers in shared memory, filled by asynchronous copies D - 1 rows
// ahead (one barrier per row).  Each thread forms the axis-C stencil at its two adjacent columns
// from 16 staged values and keeps, per column, the last NT such values in registers, from which
// the axis-B stencil gives one output row per input row.  The row loop is unrolled by D, a
// multiple of NT, so both rings are indexed by constants.
template <int NT> constexpr int plane_depth() { return NT * ((8 + NT - 1) / NT); }
// width of a ring slot of the in-plane kernel: a row's 2 nthr + NT - 1 staged inputs after its
// shift (< E elements) from a 16-byte boundary, one more value for the paired loads of an odd
// shift, rounded up to whole 16-byte chunks
template <typename T, int NT> __host__ __device__ constexpr int plane_slot(int nthr) {
    constexpr int E = 16 / sizeof(T);
    return (2 * nthr + NT + 1 + E - 1 + E - 1) / E * E;
}
template <typename T, int NT>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 4 : 3) k_lanczos_plane(const T *__restrict__ in, T *__restrict__ out, int A, int B,
                                                       int C, int L, const __grid_constant__ Taps<T> tp) {
    constexpr int D = plane_depth<NT>();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *buf = (T *)smem_raw;
    const int tid = threadIdx.x, nthr = blockDim.x;
    constexpr int E = 16 / sizeof(T);            // elements per 16-byte copy
    const int W = 2 * nthr, SW = plane_slot<T, NT>(nthr);
    const int Bo = B - (NT - 1), Co = C - (NT - 1);
    const int nrun = (Bo + L - 1) / L;
    const int a = blockIdx.y / nrun, run = blockIdx.y - a * nrun;
    const int c0 = blockIdx.x * W;
    const int b0 = run * L, b1 = min(Bo, b0 + L);
    const int nw = min(W + NT - 1, C - c0);     // staged inputs of a row segment
    const T *src = in + ((size_t)a * B + b0) * C + c0;
    T *dst = out + ((size_t)a * Bo + b0) * Co + c0 + 2 * tid;
    const bool act0 = c0 + 2 * tid < Co, act1 = c0 + 2 * tid + 1 < Co;
    const int nrow = b1 - b0 + NT - 1;
    // offset of row i's first element from a 16-byte boundary, in elements: the row is staged at
    // that offset in its slot, so a 16-byte chunk of the row lands on a 16-byte boundary
    auto shift = [&](int i) { return (int)(((uintptr_t)(src + (size_t)i * C) / sizeof(T)) % E); };
    // row i of the run into buffer `slot` (one commit group per row, empty past the run): whole
    // 16-byte chunks, and element copies for the at most 2 (E - 1) values before the first and
    // after the last chunk
    auto issue = [&](int i, int slot) {
        if (i < nrow) {
            const T *row = src + (size_t)i * C;
            const int m = shift(i);
            T *sb = buf + slot * SW + m;
            const int ja = min((E - m) % E, nw), nb = (nw - ja) / E, jt = ja + nb * E;
            for (int c = tid; c < nb; c += nthr) cp_async<16>(sb + ja + c * E, row + ja + c * E);
            const int ne = ja + (nw - jt);
            for (int e = tid; e < ne; e += nthr) {
                const int j = e < ja ? e : jt + (e - ja);
                cp_async<sizeof(T)>(sb + j, row + j);
            }
        }
        cp_async_commit();
    };
#pragma unroll
    for (int u = 0; u < D - 1; ++u) issue(u, u);
    // the last NT axis-C values of the two columns (slot = row mod NT), as one pair per row: the
    // axis-B stencil of both columns runs on pairs (FFMA2 in FP32)
    using P2 = typename std::conditional<sizeof(T) == 4, float2, double2>::type;
    P2 r[NT];
#pragma unroll
    for (int t = 0; t < NT; ++t) r[t].x = r[t].y = T(0);
    for (int i0 = 0; i0 < nrow; i0 += D) {
#pragma unroll
        for (int u = 0; u < D; ++u) {
            const int i = i0 + u;
            if (i >= nrow) break;
            cp_async_wait<D - 2>();   // row i has landed (this thread's copies)
            __syncthreads();          // every thread's copies of row i; row i - 1 is no longer read
            issue(i + D - 1, (u + D - 1) % D);
            const int m = shift(i);
            const T *sb = buf + u * SW + m + 2 * tid;
            T v[NT + 1];
            if constexpr (sizeof(T) == 4) {
                // 8-byte loads from an even offset: the row's own for an even shift, one value
                // earlier for an odd one (uniform over the CTA)
                if ((m & 1) == 0) {
#pragma unroll
                    for (int q = 0; q < (NT + 1) / 2; ++q) {
                        const float2 p2 = ((const float2 *)sb)[q];
                        v[2 * q] = p2.x, v[2 * q + 1] = p2.y;
                    }
                } else {
#pragma unroll
                    for (int q = 0; q < (NT + 3) / 2; ++q) {
                        const float2 p2 = ((const float2 *)(sb - 1))[q];
                        if (q > 0 && 2 * q - 1 <= NT) v[2 * q - 1] = p2.x;
                        if (2 * q <= NT) v[2 * q] = p2.y;
                    }
                }
            } else {
#pragma unroll
                for (int t = 0; t <= NT; ++t) v[t] = sb[t];
            }
            T x0 = T(0), x1 = T(0);
#pragma unroll
            for (int t = 0; t < NT; ++t) x0 = fma(tp.w[t], v[t], x0), x1 = fma(tp.w[t], v[t + 1], x1);
            r[u % NT].x = x0;
            r[u % NT].y = x1;
            if (i >= NT - 1) {
                P2 y;
                y.x = y.y = T(0);
#pragma unroll
                for (int t = 0; t < NT; ++t) {
                    const int sl = (u + 1 + t) % NT;   // row i - NT + 1 + t, oldest first
                    if constexpr (sizeof(T) == 4) {
                        y = __ffma2_rn(make_float2(tp.w[t], tp.w[t]), r[sl], y);
                    } else {
                        y.x = fma(tp.w[t], r[sl].x, y.x);
                        y.y = fma(tp.w[t], r[sl].y, y.y);
                    }
                }
                T *o = dst + (size_t)(i - (NT - 1)) * Co;
                if (act0) o[0] = y.x;
                if (act1) o[1] = y.y;
            }
        }
    }
    cp_async_wait<0>();
}

template <typename T, int NT>
static void sliding_passes(const T *ext, T *tmp1, T *tmp2, T *out, int d[3], const double *wd, cudaStream_t s) {
    Taps<T> tp;
    for (int i = 0; i < 64; ++i) tp.w[i] = i < NT ? (T)wd[i] : T(0);
    const int h = (NT - 1) / 2;
    // runs of L outputs along the streamed axis: long enough that the NT - 1 halo rows re-read per
    // run stay a small fraction, short enough that the grid still fills the SMs several times
    auto run_len = [&](long long cols, int A, int Bo) {
        int L = 256;
        while (L > 32 && cols * A * (long long)((Bo + L - 1) / L) < 152LL * 8 * 4) L /= 2;
        // A x runs on the grid's y axis (at most 65535)
        const int maxrun = std::max(1, 65535 / A);
        return std::max(L, (Bo + maxrun - 1) / maxrun);
    };
    // axes 2 and 1 fused: [d0][d1][d2] -> [d0][d1 - 2h][d2 - 2h]; segments of at most 512
    // outputs along C, as equal as whole warps (two outputs per thread) allow
    {
        const int Bo = d[1] - 2 * h, Co = d[2] - 2 * h;
        const int nseg = (Co + 511) / 512;
        const int per = (Co + nseg - 1) / nseg;
        const int nthr = 32 * ((per + 63) / 64);
        const int L = run_len(nseg, d[0], Bo);
        const int nrun = (Bo + L - 1) / L;
        const size_t sm = (size_t)plane_depth<NT>() * plane_slot<T, NT>(nthr) * sizeof(T);
        if (sm > 48 * 1024) cudaFuncSetAttribute(k_lanczos_plane<T, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        dim3 grid((unsigned)((Co + 2 * nthr - 1) / (2 * nthr)), (unsigned)(d[0] * nrun));
        k_lanczos_plane<T, NT><<<grid, nthr, sm, s>>>(ext, tmp1, d[0], d[1], d[2], L, tp);
        d[1] = Bo;
        d[2] = Co;
    }
    // axis 0 as the middle axis of [1][d0][d1 d2]
    {
        const int C = d[1] * d[2], Bo = d[0] - 2 * h;
        const long long nseg = (C + 255) / 256;
        const int L = run_len(nseg, 1, Bo);
        const int nrun = (Bo + L - 1) / L;
        dim3 grid((unsigned)nseg, (unsigned)nrun);
        k_lanczos_mid<T, NT><<<grid, 256, 0, s>>>(tmp1, out, 1, d[0], C, L, tp);
        d[0] = Bo;
    }
    (void)tmp2;
    count_launches(2);
}

template <typename T>
void lanczos_resample(const T *ext, T *tmp1, T *tmp2, T *out, const int cnt[3], int m, int mprime, cudaStream_t s) {
    const int h = lanczos_halo(m, mprime);
    const double rcut = (1.0 - 1.0 / m) / mprime, meff = 0.5 * m * mprime;
    int d[3] = {cnt[0] + 2 * h, cnt[1] + 2 * h, cnt[2] + 2 * h};
    double wd[64];
    lanczos_taps(h, rcut, meff, wd);
    // the strided passes put (outer index x runs) on the grid's y axis
    const bool fits = (long long)d[0] <= 65535;
    switch (fits ? 2 * h + 1 : 0) {
        case 3: sliding_passes<T, 3>(ext, tmp1, tmp2, out, d, wd, s); return;
        case 5: sliding_passes<T, 5>(ext, tmp1, tmp2, out, d, wd, s); return;
        case 7: sliding_passes<T, 7>(ext, tmp1, tmp2, out, d, wd, s); return;
        case 9: sliding_passes<T, 9>(ext, tmp1, tmp2, out, d, wd, s); return;
        case 11: sliding_passes<T, 11>(ext, tmp1, tmp2, out, d, wd, s); return;
        case 13: sliding_passes<T, 13>(ext, tmp1, tmp2, out, d, wd, s); return;
        case 15: sliding_passes<T, 15>(ext, tmp1, tmp2, out, d, wd, s); return;
        case 17: sliding_passes<T, 17>(ext, tmp1, tmp2, out, d, wd, s); return;
        default: break;
    }
    // wider stencils: one thread per output voxel
    const size_t sm = (2 * h + 1) * sizeof(T);
    auto launch = [&](const T *a, T *b, int axis) {
        size_t tot = (size_t)d[0] * d[1] * d[2];
        tot = tot / d[axis] * (d[axis] - 2 * h);
        unsigned nb = (unsigned)std::min<size_t>((tot + 255) / 256, 152 * 16);
        k_lanczos_axis<T><<<std::max(1u, nb), 256, sm, s>>>(a, b, d[0], d[1], d[2], axis, h, rcut, meff);
        count_launches(1);
        d[axis] -= 2 * h;
    };
    launch(ext, tmp1, 2);
    launch(tmp1, tmp2, 1);
    launch(tmp2, out, 0);
}

// Spherical cutoff (not separable): one thread per output voxel, (2h+1)^3 taps with the
// normalised weights staged in shared memory; consecutive threads take consecutive voxels of a
// row, so every tap is a coalesced read of the halo-extended volume.
template <typename T>
__global__ void k_sphere_stencil(const T *__restrict__ ext, const T *__restrict__ wg, T *__restrict__ out, int c0,
                                 int c1, int c2, int h) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *w = (T *)smem_raw;
    const int nt = 2 * h + 1, nt3 = nt * nt * nt;
    for (int i = threadIdx.x; i < nt3; i += blockDim.x) w[i] = wg[i];
    __syncthreads();
    const int e1 = c1 + 2 * h, e2 = c2 + 2 * h;
    const size_t total = (size_t)c0 * c1 * c2;
    for (size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x; v < total; v += (size_t)gridDim.x * blockDim.x) {
        const int i2 = (int)(v % c2), i1 = (int)((v / c2) % c1), i0 = (int)(v / ((size_t)c2 * c1));
        T acc = T(0);
        for (int t0 = 0; t0 < nt; ++t0)
            for (int t1 = 0; t1 < nt; ++t1) {
                const T *row = ext + ((size_t)(i0 + t0) * e1 + (i1 + t1)) * e2 + i2;
                const T *wr = w + (t0 * nt + t1) * nt;
                for (int t2 = 0; t2 < nt; ++t2) acc = fma(wr[t2], row[t2], acc);
            }
        out[v] = acc;
    }
}

template <typename T>
void sphere_resample(const T *ext, const T *w, T *out, const int cnt[3], int h, cudaStream_t s) {
    const size_t tot = (size_t)cnt[0] * cnt[1] * cnt[2];
    const int nt = 2 * h + 1;
    const size_t sm = (size_t)nt * nt * nt * sizeof(T);
    if (sm > 48 * 1024) cudaFuncSetAttribute(k_sphere_stencil<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    const unsigned nb = (unsigned)std::max<size_t>(1, std::min<size_t>((tot + 255) / 256, 152 * 16));
    k_sphere_stencil<T><<<nb, 256, sm, s>>>(ext, w, out, cnt[0], cnt[1], cnt[2], h);
    count_launches(1);
}

template void sphere_resample<float>(const float *, const float *, float *, const int *, int, cudaStream_t);
template void sphere_resample<double>(const double *, const double *, double *, const int *, int, cudaStream_t);
template void lanczos_resample<float>(const float *, float *, float *, float *, const int *, int, int, cudaStream_t);
template void lanczos_resample<double>(const double *, double *, double *, double *, const int *, int, int,
                                       cudaStream_t);

}  // namespace ds
