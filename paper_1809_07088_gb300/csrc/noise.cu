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
// to 17 taps run as sliding windows (each input read about once per pass: HBM bound); wider
// ones with one thread per output.
#include <algorithm>

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
// read about (L + NT - 1) / L times; consecutive threads take consecutive c (coalesced).
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
    for (int b = b0; b < b1; ++b) {
        ring[NT - 1] = src[(size_t)(b - b0 + NT - 1) * C];
        T acc = T(0);
#pragma unroll
        for (int t = 0; t < NT; ++t) acc = fma(tp.w[t], ring[t], acc);
        dst[(size_t)(b - b0) * C] = acc;
#pragma unroll
        for (int t = 0; t < NT - 1; ++t) ring[t] = ring[t + 1];
    }
}

// Pass along the contiguous axis of [R][C]: a block stages a row segment and its halo in shared
// memory (coalesced), then each thread forms outputs from the staged values.
template <typename T, int NT>
__global__ void __launch_bounds__(256) k_lanczos_row(const T *__restrict__ in, T *__restrict__ out, int C, int SEG,
                                                     const __grid_constant__ Taps<T> tp) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *seg = (T *)smem_raw;
    const int Co = C - (NT - 1);
    const int nseg = (Co + SEG - 1) / SEG;
    const size_t r = blockIdx.x / nseg;
    const int s0 = (int)(blockIdx.x - r * nseg) * SEG;
    const int n = min(SEG, Co - s0);
    const T *src = in + r * C + s0;
    for (int i = threadIdx.x; i < n + NT - 1; i += blockDim.x) seg[i] = src[i];
    __syncthreads();
    T *dst = out + r * Co + s0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        T acc = T(0);
#pragma unroll
        for (int t = 0; t < NT; ++t) acc = fma(tp.w[t], seg[i + t], acc);
        dst[i] = acc;
    }
}

template <typename T, int NT>
static void sliding_passes(const T *ext, T *tmp1, T *tmp2, T *out, int d[3], const double *wd, cudaStream_t s) {
    Taps<T> tp;
    for (int i = 0; i < 64; ++i) tp.w[i] = i < NT ? (T)wd[i] : T(0);
    const int h = (NT - 1) / 2;
    // axis 2 (contiguous): rows of d2, segments of up to 2048 outputs
    {
        const size_t R = (size_t)d[0] * d[1];
        const int Co = d[2] - 2 * h, SEG = std::min(Co, 2048);
        const size_t nb = R * (size_t)((Co + SEG - 1) / SEG);
        k_lanczos_row<T, NT><<<(unsigned)nb, 256, (SEG + NT - 1) * sizeof(T), s>>>(ext, tmp1, d[2], SEG, tp);
        d[2] = Co;
    }
    // axis 1: [d0][d1][d2], then axis 0: [1][d0][d1 d2]; runs of L outputs per thread
    auto mid = [&](const T *a, T *b, int A, int B, int C) {
        // runs of at least 64 outputs, longer when A x runs would exceed the grid's y limit
        const int Bo = B - 2 * h;
        const int L = std::max(64, (int)(((long long)Bo * A + 65534) / 65535));
        const int nrun = (Bo + L - 1) / L;
        dim3 grid((unsigned)((C + 255) / 256), (unsigned)(A * nrun));
        k_lanczos_mid<T, NT><<<grid, 256, 0, s>>>(a, b, A, B, C, L, tp);
    };
    mid(tmp1, tmp2, d[0], d[1], d[2]);
    d[1] -= 2 * h;
    mid(tmp2, out, 1, d[0], d[1] * d[2]);
    d[0] -= 2 * h;
    count_launches(3);
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
