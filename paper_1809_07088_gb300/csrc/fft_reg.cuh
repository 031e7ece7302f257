// Register-resident line FFTs of compile-time length N (mixed radix 4, 2, 3, 5, 7), sign +i,
// unnormalised, as in Eq. (fft) of Section III A:  X_k = sum_R x_R exp(+2 pi i k R / N).
//
// A line lives in one thread's registers; the Stockham passes are unrolled at compile time, so
// every element index and every twiddle factor is a constant: the twiddles exp(2 pi i m / N) are
// computed by the compiler (below) and enter the code as immediate operands, with no table.
#pragma once

#include <utility>

#include "ds_common.cuh"
#include "fft_lines.cuh"

namespace ds {

// ---- compile-time roots of unity --------------------------------------------------------------
// cos and sin of 2 pi m / n: the angle is reduced exactly in integers to an octant q and a
// remainder phi in [0, pi/4) (or its complement pi/4 - phi), whose sine and cosine are summed from
// their Taylor series (13 terms: the first omitted term is below 1e-27 for |x| <= pi/4).
constexpr double kRootPi = 3.14159265358979323846264338327950288;
constexpr double taylor_sin(double x) {
    double x2 = x * x, t = x, s = x;
    for (int k = 1; k <= 13; ++k) {
        t *= -x2 / ((2.0 * k) * (2.0 * k + 1.0));
        s += t;
    }
    return s;
}
constexpr double taylor_cos(double x) {
    double x2 = x * x, t = 1.0, s = 1.0;
    for (int k = 1; k <= 13; ++k) {
        t *= -x2 / ((2.0 * k - 1.0) * (2.0 * k));
        s += t;
    }
    return s;
}
// which = 0: cosine, 1: sine of 2 pi m / n
constexpr double root_cs(int n, int m, int which) {
    const int r = ((m % n) + n) % n;
    const int e = 8 * r, q = e / n, rem = e - q * n;
    const double phi = kRootPi * rem / (4.0 * n);          // [0, pi/4)
    const double psi = kRootPi * (n - rem) / (4.0 * n);    // pi/4 - phi, (0, pi/4]
    double c = 0.0, s = 0.0;
    switch (q) {
        case 0: c = taylor_cos(phi), s = taylor_sin(phi); break;
        case 1: c = taylor_sin(psi), s = taylor_cos(psi); break;
        case 2: c = -taylor_sin(phi), s = taylor_cos(phi); break;
        case 3: c = -taylor_cos(psi), s = taylor_sin(psi); break;
        case 4: c = -taylor_cos(phi), s = -taylor_sin(phi); break;
        case 5: c = -taylor_sin(psi), s = -taylor_cos(psi); break;
        case 6: c = taylor_sin(phi), s = -taylor_cos(phi); break;
        default: c = taylor_cos(psi), s = -taylor_sin(psi); break;
    }
    return which ? s : c;
}

// compile-time loop: f(std::integral_constant<int, I>) for I in [B, E)
template <int B, int E> struct StaticFor {
    template <class F> __device__ __forceinline__ static void run(F &&f) {
        if constexpr (B < E) {
            f(std::integral_constant<int, B>{});
            StaticFor<B + 1, E>::run(f);
        }
    }
};

constexpr int reg_radix(int rem) {
    return rem % 4 == 0 ? 4 : rem % 2 == 0 ? 2 : rem % 3 == 0 ? 3 : rem % 5 == 0 ? 5 : 7;
}
constexpr bool reg_fft_size(int n) {
    int m = n;
    for (int r : {4, 2, 3, 5, 7})
        while (m % r == 0) m /= r;
    return m == 1 && n >= 1;
}

// In-place transform of a[0..N) (registers).  Stockham pass of radix R at stride Ns: read R elements
// N/R apart, twiddle by w^(k r N/(Ns R)), k = j mod Ns, R-point DFT, write them Ns apart.
template <typename T, int N> struct RegFFT {
    using C = c_t<T>;
    template <int NS, int REM> __device__ __forceinline__ static void pass(C (&a)[N]) {
        if constexpr (REM > 1) {
            constexpr int R = reg_radix(REM);
            constexpr int NR = N / R;
            constexpr int TWS = N / (NS * R);
            C b[N];
            StaticFor<0, NR>::run([&](auto jc) {
                constexpr int j = decltype(jc)::value;
                constexpr int k = j % NS;
                C v[R];
                StaticFor<0, R>::run([&](auto rc) {
                    constexpr int r = decltype(rc)::value;
                    C x = a[j + r * NR];
                    constexpr int m = (k * r * TWS) % N;
                    if constexpr (m != 0) {
                        constexpr T wc = (T)root_cs(N, m, 0), ws = (T)root_cs(N, m, 1);
                        x = cmul(x, mk<T>(wc, ws));
                    }
                    v[r] = x;
                });
                dft_small<C, T>(v, R);
                constexpr int idxD = (j - k) * R + k;
                StaticFor<0, R>::run([&](auto rc) {
                    constexpr int r = decltype(rc)::value;
                    b[idxD + r * NS] = v[r];
                });
            });
#pragma unroll
            for (int i = 0; i < N; ++i) a[i] = b[i];
            pass<NS * R, REM / R>(a);
        }
    }
    __device__ __forceinline__ static void run(C (&a)[N]) { pass<1, N>(a); }
};

}  // namespace ds
