// Noise reduction (Section V).
//
// Lanczos resampling on the commensurate grid (Section V B): for Q on the supercell Bragg
// grid, Eq. (intensity_convol_finite) with W = W_sinc L (Eqs. weight_sinc, windowed_sinc,
// lanczos) separates into three one-axis passes, each a (2h+1)-tap stencil with weights
//     w(d) = sinc(2 pi r_cut d) sinc(pi d / m_eff),  |d| < m_eff,
// normalised to unit sum (the 8 r_cut^3 prefactor and the denominator of Eq.
// intensity_convol_finite both cancel in the normalisation).  r_cut = (1 - 1/m)/m' and
// m_eff = m m' / 2 (m' = 2 is the plain window; larger m' reaches zero at 1/m').  Each pass
// shrinks the volume by the halo h = ceil(m_eff) - 1 on both sides of its axis.
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

template <typename T>
void lanczos_resample(const T *ext, T *tmp1, T *tmp2, T *out, const int cnt[3], int m, int mprime, cudaStream_t s) {
    const int h = lanczos_halo(m, mprime);
    const double rcut = (1.0 - 1.0 / m) / mprime, meff = 0.5 * m * mprime;
    int d[3] = {cnt[0] + 2 * h, cnt[1] + 2 * h, cnt[2] + 2 * h};
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

template void lanczos_resample<float>(const float *, float *, float *, float *, const int *, int, int, cudaStream_t);
template void lanczos_resample<double>(const double *, double *, double *, double *, const int *, int, int,
                                       cudaStream_t);

}  // namespace ds
