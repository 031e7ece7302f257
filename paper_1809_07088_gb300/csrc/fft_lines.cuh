// Mixed-radix (2, 3, 4, 5, 7) self-sorting Stockham FFT over batches of lines that sit in
// shared memory.  Sign +i and no normalisation, as in Eq. (fft) of Section III A:
//     X_k = sum_R x_R exp(+2 pi i k R / n).
//
// A pass of radix r reads r elements a stride n/r apart, applies the twiddles
// w^(k r n/(Ns r)) with w = exp(2 pi i / n) taken from a table of the n roots of unity
// (generated in FP64), does an r-point DFT in registers and writes the r results Ns apart
// into the other buffer; Ns grows by r each pass and the last pass leaves the transform in
// natural order.  All lines of the batch are processed together, one butterfly per thread per
// task, so the CTA stays busy whatever the line count.
#pragma once

#include "ds_common.cuh"

namespace ds {

// Exact x / d for x d < 2^32 by a high multiply: m = ceil(2^32 / d) (0 stands for d = 1); with
// x = q d + r, x m / 2^32 = q + (r + x e / 2^32) / d, e = m d - 2^32 < d, and x e < x d < 2^32
// keeps the fraction below 1.  The FFT index arithmetic (counts below 2^24 whose products with
// their divisors stay below 2^32 for supercells of up to 128 cells per axis) uses it instead of
// integer division; the per-pass divisors come with the axis plan, built on the host.
struct FastDiv {
    unsigned d, m;
    __host__ __device__ __forceinline__ static unsigned magic(unsigned dd) { return dd == 1 ? 0u : 0xFFFFFFFFu / dd + 1u; }
    __host__ __device__ __forceinline__ FastDiv(unsigned dd, unsigned mm) : d(dd), m(mm) {}
    __host__ __device__ __forceinline__ explicit FastDiv(unsigned dd) : d(dd), m(magic(dd)) {}
    __device__ __forceinline__ unsigned div(unsigned x) const { return m ? __umulhi(x, m) : x; }
};

struct AxisPlan {
    int n;       // transform length
    int nrad;    // number of radix passes
    int rad[8];  // radices in pass order
    unsigned mNR[8], mNs[8];  // FastDiv magics of n / rad[p] and of the running product Ns before pass p
};


template <typename C, typename T> __device__ __forceinline__ void dft_small(C *v, int R) {
    // r-point DFT with the +i sign, in place
    if (R == 2) {
        C t = v[0];
        v[0] = cadd(t, v[1]);
        v[1] = csub(t, v[1]);
    } else if (R == 4) {
        C t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
        C t2 = cadd(v[1], v[3]), t3 = csub(v[1], v[3]);
        C it3 = mk<T>(-t3.y, t3.x);
        v[0] = cadd(t0, t2);
        v[2] = csub(t0, t2);
        v[1] = cadd(t1, it3);
        v[3] = csub(t1, it3);
    } else if (R == 3) {
        const T s = T(0.86602540378443864676372317075294);  // sin(2 pi / 3)
        C t1 = cadd(v[1], v[2]);
        C t2 = mk<T>(v[0].x - T(0.5) * t1.x, v[0].y - T(0.5) * t1.y);
        C d = csub(v[1], v[2]);
        C t3 = mk<T>(-s * d.y, s * d.x);  // i s (a1 - a2)
        v[0] = cadd(v[0], t1);
        v[1] = cadd(t2, t3);
        v[2] = csub(t2, t3);
    } else if (R == 5) {
        const T c1 = T(0.30901699437494742410229341718282);   // cos(2 pi/5)
        const T c2 = T(-0.80901699437494742410229341718282);  // cos(4 pi/5)
        const T s1 = T(0.95105651629515357211643933337938);   // sin(2 pi/5)
        const T s2 = T(0.58778525229247312916870595463907);   // sin(4 pi/5)
        C p14 = cadd(v[1], v[4]), m14 = csub(v[1], v[4]);
        C p23 = cadd(v[2], v[3]), m23 = csub(v[2], v[3]);
        C a = v[0];
        C r1 = mk<T>(a.x + c1 * p14.x + c2 * p23.x, a.y + c1 * p14.y + c2 * p23.y);
        C r2 = mk<T>(a.x + c2 * p14.x + c1 * p23.x, a.y + c2 * p14.y + c1 * p23.y);
        C i1 = mk<T>(s1 * m14.x + s2 * m23.x, s1 * m14.y + s2 * m23.y);
        C i2 = mk<T>(s2 * m14.x - s1 * m23.x, s2 * m14.y - s1 * m23.y);
        v[0] = mk<T>(a.x + p14.x + p23.x, a.y + p14.y + p23.y);
        v[1] = mk<T>(r1.x - i1.y, r1.y + i1.x);  // r1 + i * i1
        v[4] = mk<T>(r1.x + i1.y, r1.y - i1.x);  // r1 - i * i1
        v[2] = mk<T>(r2.x - i2.y, r2.y + i2.x);
        v[3] = mk<T>(r2.x + i2.y, r2.y - i2.x);
    } else {  // R == 7: direct small DFT
        const T cs[7] = {T(1), T(0.62348980185873353052500488400424), T(-0.22252093395631440428890256449680),
                         T(-0.90096886790241912623610231950745), T(-0.90096886790241912623610231950745),
                         T(-0.22252093395631440428890256449680), T(0.62348980185873353052500488400424)};
        const T sn[7] = {T(0), T(0.78183148246802980870844452667406), T(0.97492791218182360701813168299393),
                         T(0.43388373911755812047576833284836), T(-0.43388373911755812047576833284836),
                         T(-0.97492791218182360701813168299393), T(-0.78183148246802980870844452667406)};
        C out[7];
#pragma unroll
        for (int q = 0; q < 7; ++q) {
            C acc = v[0];
#pragma unroll
            for (int r = 1; r < 7; ++r) {
                const int e = (r * q) % 7;
                acc.x += cs[e] * v[r].x - sn[e] * v[r].y;
                acc.y += cs[e] * v[r].y + sn[e] * v[r].x;
            }
            out[q] = acc;
        }
#pragma unroll
        for (int q = 0; q < 7; ++q) v[q] = out[q];
    }
}

// One Stockham pass of compile-time radix R over every line of the batch (see fft_lines).
template <typename T, int R>
__device__ __forceinline__ void radix_pass(const c_t<T> *__restrict__ a, c_t<T> *__restrict__ b, const c_t<T> *W,
                                           int NR, int Ns, int tw, int nlines, int inner_stride, int outer_stride,
                                           int estride, bool j_fast, const FastDiv &fNR, const FastDiv &fNs,
                                           const FastDiv &flines, const FastDiv &finner) {
    using C = c_t<T>;
    const int tasks = nlines * NR;
    const int inner = (int)finner.d;
    for (int task = threadIdx.x; task < tasks; task += blockDim.x) {
        int L, j;
        if (j_fast) {
            L = (int)fNR.div((unsigned)task);
            j = task - L * NR;
        } else {
            j = (int)flines.div((unsigned)task);
            L = task - j * nlines;
        }
        const int Lo = (int)finner.div((unsigned)L);
        const int base = Lo * outer_stride + (L - Lo * inner) * inner_stride;
        const int k = j - (int)fNs.div((unsigned)j) * Ns;
        C v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            C x = a[base + (j + r * NR) * estride];
            // k r tw < Ns R tw = n: the root index needs no reduction
            if (r > 0) x = cmul(x, W[k * r * tw]);
            v[r] = x;
        }
        dft_small<C, T>(v, R);
        const int idxD = (j - k) * R + k;  // (j / Ns) Ns R + k
#pragma unroll
        for (int r = 0; r < R; ++r) b[base + (idxD + r * Ns) * estride] = v[r];
    }
}

// Transform nlines lines of length P.n.  Element e of line L lives at
//     (L / inner) * outer_stride + (L % inner) * inner_stride + e * estride
// in buffer `a`; `b` is a same-sized scratch buffer.  Returns the buffer that holds the result.
// Must be called by every thread of the block (contains __syncthreads).
template <typename T>
__device__ c_t<T> *fft_lines(c_t<T> *a, c_t<T> *b, const AxisPlan &P, const c_t<T> *W, int nlines,
                             int inner, int inner_stride, int outer_stride, int estride) {
    using C = c_t<T>;
    const int n = P.n;
    int Ns = 1;
    const bool j_fast = (estride == 1);
    const FastDiv finner((unsigned)inner), flines((unsigned)nlines);
    for (int p = 0; p < P.nrad; ++p) {
        const int R = P.rad[p];
        const int NR = n / R;
        const int tw = n / (Ns * R);
        const FastDiv fNR((unsigned)NR, P.mNR[p]), fNs((unsigned)Ns, P.mNs[p]);
        switch (R) {
        case 4: radix_pass<T, 4>(a, b, W, NR, Ns, tw, nlines, inner_stride, outer_stride, estride, j_fast, fNR, fNs, flines, finner); break;
        case 2: radix_pass<T, 2>(a, b, W, NR, Ns, tw, nlines, inner_stride, outer_stride, estride, j_fast, fNR, fNs, flines, finner); break;
        case 3: radix_pass<T, 3>(a, b, W, NR, Ns, tw, nlines, inner_stride, outer_stride, estride, j_fast, fNR, fNs, flines, finner); break;
        case 5: radix_pass<T, 5>(a, b, W, NR, Ns, tw, nlines, inner_stride, outer_stride, estride, j_fast, fNR, fNs, flines, finner); break;
        default: radix_pass<T, 7>(a, b, W, NR, Ns, tw, nlines, inner_stride, outer_stride, estride, j_fast, fNR, fNs, flines, finner); break;
        }
        __syncthreads();
        C *t = a;
        a = b;
        b = t;
        Ns *= R;
    }
    return a;
}

}  // namespace ds
