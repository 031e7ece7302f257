// Batched 3D real-to-half-complex FFT of per-site lattice fields (Eqs. fft, comp_ft, mag_ft,
// U_fft, A_fft of Section III), unnormalised, sign +i.
//
// Pass 1 (planes): one CTA loads `ppc` consecutive R1-planes of one field.  The field values
// are generated on the fly from the model arrays (occupancy deviation, moment component, or
// Taylor monomial w u~x^a u~y^b u~z^c / (a! b! c!) built from per-atom power tables), rows
// R2 = 2p and 2p+1 are packed as one complex line, transformed along axis 3, split into the
// two half spectra (Hermitian separation), and the half-width plane is transformed along
// axis 2.  The plane goes to the work buffer [field][R1][k2][k3h].
// Pass 2 (columns): one CTA loads `cb` consecutive (k2, k3h) columns of one field, transforms
// them along axis 1 and writes the half spectrum [field][k1][k2][k3h], multiplied by i^n for
// displacive monomials of order n.  All global traffic is contiguous runs.
// Large batches of small fields (whole field in shared memory) take one kernel for all three axes.
#include <algorithm>

#include "fft_reg.cuh"
#include "internal.h"

namespace ds {

template <typename T> __global__ void k_twiddles(int n, c_t<T> *W) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    double s, c;
    sincospi(2.0 * (double)e / (double)n, &s, &c);
    W[e] = mk<T>((T)c, (T)s);
}

template <typename T> void make_twiddles(int n, c_t<T> *W, cudaStream_t s) {
    k_twiddles<T><<<(n + 127) / 128, 128, 0, s>>>(n, W);
    count_launches(1);
}

// The rows of model data that make up real field f, resolved once per CTA so that the per-cell
// value is a few loads and multiplies (no division by the field counts in the load loops).
template <typename T> struct FieldRow {
    int kind;
    const uint8_t *occ;  // occupancy row (SRC_OCC; SRC_DISP weights, may be null)
    const float *vec;    // moment row, component `comp` (SRC_SPIN)
    const T *pw[3];      // power rows (u_a Q_s)^e_a / e_a! (SRC_DISP)
    const T *real;       // SRC_REAL row
    int comp;
    T mean;              // subtracted site mean (SRC_OCC / SRC_SPIN, DIFFUSE), else 0
};

template <typename T> __device__ __forceinline__ FieldRow<T> field_row(const FieldSource &src, int ncell, int f) {
    FieldRow<T> r;
    r.kind = src.kind;
    r.occ = nullptr;
    r.vec = nullptr;
    r.pw[0] = r.pw[1] = r.pw[2] = nullptr;
    r.real = nullptr;
    r.comp = 0;
    r.mean = T(0);
    const int m = f / src.nf_per_model;
    const int lf = f - m * src.nf_per_model;
    switch (src.kind) {
    case SRC_OCC:
        r.occ = src.occ + ((size_t)m * src.nsite + lf) * ncell;
        if (src.diffuse) r.mean = (T)src.mean[lf];
        break;
    case SRC_SPIN: {
        const int mu = lf / 3, a = lf - 3 * mu;
        r.vec = src.vec3 + ((size_t)m * src.nsite + mu) * ncell * 3;
        r.comp = a;
        if (src.diffuse) r.mean = (T)src.mean[mu * 3 + a];
        break;
    }
    case SRC_DISP: {
        const int mu = lf / src.T, t = lf - mu * src.T;
        const int4 e = src.terms[t];
        const size_t P1 = (size_t)src.P + 1;
        const T *base = (const T *)src.pw + (((size_t)m * src.nsite + mu) * 3) * P1 * ncell;
        r.pw[0] = base + (0 * P1 + e.x) * ncell;
        r.pw[1] = base + (1 * P1 + e.y) * ncell;
        r.pw[2] = base + (2 * P1 + e.z) * ncell;
        if (src.occ) r.occ = src.occ + ((size_t)m * src.nsite + mu) * ncell;
        break;
    }
    default:
        r.real = (const T *)src.real_buf + (size_t)f * ncell;
    }
    return r;
}

// value of the field at lattice point `cell` (linear [R1][R2][R3])
template <typename T> __device__ __forceinline__ T row_value(const FieldRow<T> &r, int cell) {
    switch (r.kind) {
    case SRC_OCC: return (T)r.occ[cell] - r.mean;
    case SRC_SPIN: return (T)r.vec[(size_t)cell * 3 + r.comp] - r.mean;
    case SRC_DISP: {
        T v = r.pw[0][cell] * r.pw[1][cell] * r.pw[2][cell];
        if (r.occ) v *= (T)r.occ[cell];
        return v;
    }
    default: return r.real[cell];
    }
}

template <typename T>
__global__ void k_fft_planes(Geometry g, FieldSource src, int f0, int ppc, c_t<T> *work, const c_t<T> *W2g,
                             const c_t<T> *W3g) {
    using C = c_t<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n1 = g.n[0], n2 = g.n[1], n3 = g.n[2], n3h = g.n3h;
    const int n2p = (n2 + 1) / 2;
    const int plane_c = n2p * n3 > n2 * n3h ? n2p * n3 : n2 * n3h;
    C *W2 = (C *)smem_raw;
    C *W3 = W2 + n2;
    C *bufA = W3 + n3;
    C *bufB = bufA + (size_t)ppc * plane_c;
    for (int i = threadIdx.x; i < n2; i += blockDim.x) W2[i] = W2g[i];
    for (int i = threadIdx.x; i < n3; i += blockDim.x) W3[i] = W3g[i];

    const int nchunk = (g.n[0] + ppc - 1) / ppc;
    const int fl = blockIdx.x / nchunk;
    const int f = f0 + fl;
    const int r1_0 = (blockIdx.x - fl * nchunk) * ppc;
    const int np = min(ppc, n1 - r1_0);
    const int ncell = g.ncell;
    const FieldRow<T> fr = field_row<T>(src, ncell, f);

    // load: complex line p of plane q holds rows 2p (real) and 2p + 1 (imaginary)
    const int per_plane_in = n2p * n3;
    const FastDiv fin((unsigned)per_plane_in), f3((unsigned)n3), fh((unsigned)n3h), fph((unsigned)(n2 * n3h));
    for (int idx = threadIdx.x; idx < np * per_plane_in; idx += blockDim.x) {
        const int q = (int)fin.div((unsigned)idx), rem = idx - q * per_plane_in;
        const int p = (int)f3.div((unsigned)rem), r3 = rem - p * n3;
        const int cell0 = ((r1_0 + q) * n2 + 2 * p) * n3 + r3;
        const T x = row_value<T>(fr, cell0);
        const T y = (2 * p + 1 < n2) ? row_value<T>(fr, cell0 + n3) : T(0);
        bufA[(size_t)q * plane_c + p * n3 + r3] = mk<T>(x, y);
    }
    __syncthreads();
    // axis 3: np * n2p contiguous lines (plane stride plane_c)
    C *res = fft_lines<T>(bufA, bufB, g.ax[2], W3, np * n2p, n2p, n3, plane_c, 1);
    C *dst = (res == bufA) ? bufB : bufA;
    // separate the packed rows: X = (Z + conj Z-)/2, Y = (Z - conj Z-)/(2i), keep k3 < n3h
    const int per_plane_h = n2 * n3h;
    for (int idx = threadIdx.x; idx < np * per_plane_h; idx += blockDim.x) {
        const int q = (int)fph.div((unsigned)idx), rem = idx - q * per_plane_h;
        const int row = (int)fh.div((unsigned)rem), k3 = rem - row * n3h;
        const int p = row >> 1;
        const C z = res[(size_t)q * plane_c + p * n3 + k3];
        const C zm = res[(size_t)q * plane_c + p * n3 + (k3 == 0 ? 0 : n3 - k3)];
        C v;
        if ((row & 1) == 0)
            v = mk<T>(T(0.5) * (z.x + zm.x), T(0.5) * (z.y - zm.y));
        else
            v = mk<T>(T(0.5) * (z.y + zm.y), T(-0.5) * (z.x - zm.x));
        dst[(size_t)q * plane_c + row * n3h + k3] = v;
    }
    __syncthreads();
    // axis 2: np * n3h lines of stride n3h
    C *res2 = fft_lines<T>(dst, res, g.ax[1], W2, np * n3h, n3h, 1, plane_c, n3h);
    C *out = work + ((size_t)fl * n1 + r1_0) * per_plane_h;
    for (int idx = threadIdx.x; idx < np * per_plane_h; idx += blockDim.x) {
        const int q = (int)fph.div((unsigned)idx), rem = idx - q * per_plane_h;
        out[(size_t)q * per_plane_h + rem] = res2[(size_t)q * plane_c + rem];
    }
}

template <typename T>
__global__ void k_fft_columns(Geometry g, FieldSource src, int f0, int cb, const c_t<T> *work, c_t<T> *spec,
                              const c_t<T> *W1g) {
    using C = c_t<T>;
    griddep_launch_dependents();   // the consumer of the spectra may be scheduled
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n1 = g.n[0];
    const int ncol = g.n[1] * g.n3h;
    C *W1 = (C *)smem_raw;
    C *bufA = W1 + n1;
    C *bufB = bufA + (size_t)n1 * cb;
    for (int i = threadIdx.x; i < n1; i += blockDim.x) W1[i] = W1g[i];
    const int nchunk = (ncol + cb - 1) / cb;
    const int fl = blockIdx.x / nchunk;
    const int f = f0 + fl;
    const int c0 = (blockIdx.x - fl * nchunk) * cb;
    const C *in = work + (size_t)fl * n1 * ncol;
    const FastDiv fcb((unsigned)cb);
    for (int idx = threadIdx.x; idx < n1 * cb; idx += blockDim.x) {
        const int r1 = (int)fcb.div((unsigned)idx), c = idx - r1 * cb;
        bufA[idx] = (c0 + c < ncol) ? in[(size_t)r1 * ncol + c0 + c] : mk<T>(T(0), T(0));
    }
    __syncthreads();
    C *res = fft_lines<T>(bufA, bufB, g.ax[0], W1, cb, cb, 1, 0, cb);
    int rot = 0;
    if (src.kind == SRC_DISP) {
        const int lf = f % src.nf_per_model;
        rot = src.terms[lf % src.T].w;
    }
    C *out = spec + (size_t)f * g.ncell_h;
    for (int idx = threadIdx.x; idx < n1 * cb; idx += blockDim.x) {
        const int k1 = (int)fcb.div((unsigned)idx), c = idx - k1 * cb;
        if (c0 + c < ncol) out[(size_t)k1 * ncol + c0 + c] = cipow(res[idx], rot);
    }
}

// Whole-field variant for small supercells: one CTA holds every plane of one field in shared
// memory and runs the three axes back to back (axis 3 with row packing and Hermitian
// separation, axis 2, then axis 1 over the plane stride), writing the half spectrum once.  Same
// arithmetic as the two-pass kernels, without the work buffer round trip.
template <typename T>
__global__ void __launch_bounds__(512) k_fft_field(Geometry g, FieldSource src, int f0, c_t<T> *spec,
                                                   const c_t<T> *W1g, const c_t<T> *W2g, const c_t<T> *W3g) {
    using C = c_t<T>;
    griddep_launch_dependents();   // the consumer of the spectra may be scheduled
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n1 = g.n[0], n2 = g.n[1], n3 = g.n[2], n3h = g.n3h;
    const int n2p = (n2 + 1) / 2;
    const int plane_c = n2p * n3 > n2 * n3h ? n2p * n3 : n2 * n3h;
    C *W1 = (C *)smem_raw;
    C *W2 = W1 + n1;
    C *W3 = W2 + n2;
    C *bufA = W3 + n3;
    C *bufB = bufA + (size_t)n1 * plane_c;
    for (int i = threadIdx.x; i < n1; i += blockDim.x) W1[i] = W1g[i];
    for (int i = threadIdx.x; i < n2; i += blockDim.x) W2[i] = W2g[i];
    for (int i = threadIdx.x; i < n3; i += blockDim.x) W3[i] = W3g[i];
    const int f = f0 + blockIdx.x;
    const int ncell = g.ncell;
    const FieldRow<T> fr = field_row<T>(src, ncell, f);
    const int per_plane_in = n2p * n3;
    const int per_plane_h = n2 * n3h;
    const FastDiv fin((unsigned)per_plane_in), f3((unsigned)n3), fh((unsigned)n3h), fph((unsigned)per_plane_h);
    for (int idx = threadIdx.x; idx < n1 * per_plane_in; idx += blockDim.x) {
        const int q = (int)fin.div((unsigned)idx), rem = idx - q * per_plane_in;
        const int pr = (int)f3.div((unsigned)rem), r3 = rem - pr * n3;
        const int cell0 = (q * n2 + 2 * pr) * n3 + r3;
        const T x = row_value<T>(fr, cell0);
        const T y = (2 * pr + 1 < n2) ? row_value<T>(fr, cell0 + n3) : T(0);
        bufA[(size_t)q * plane_c + pr * n3 + r3] = mk<T>(x, y);
    }
    __syncthreads();
    C *res = fft_lines<T>(bufA, bufB, g.ax[2], W3, n1 * n2p, n2p, n3, plane_c, 1);
    C *dst = (res == bufA) ? bufB : bufA;
    for (int idx = threadIdx.x; idx < n1 * per_plane_h; idx += blockDim.x) {
        const int q = (int)fph.div((unsigned)idx), rem = idx - q * per_plane_h;
        const int row = (int)fh.div((unsigned)rem), k3 = rem - row * n3h;
        const int pr = row >> 1;
        const C z = res[(size_t)q * plane_c + pr * n3 + k3];
        const C zm = res[(size_t)q * plane_c + pr * n3 + (k3 == 0 ? 0 : n3 - k3)];
        C v;
        if ((row & 1) == 0)
            v = mk<T>(T(0.5) * (z.x + zm.x), T(0.5) * (z.y - zm.y));
        else
            v = mk<T>(T(0.5) * (z.y + zm.y), T(-0.5) * (z.x - zm.x));
        dst[(size_t)q * plane_c + row * n3h + k3] = v;
    }
    __syncthreads();
    C *res2 = fft_lines<T>(dst, res, g.ax[1], W2, n1 * n3h, n3h, 1, plane_c, n3h);
    C *oth = (res2 == bufA) ? bufB : bufA;
    // axis 1: line L = (k2, k3) at offset L, element r1 at r1 * plane_c
    C *res3 = fft_lines<T>(res2, oth, g.ax[0], W1, per_plane_h, per_plane_h, 1, 0, plane_c);
    int rot = 0;
    if (src.kind == SRC_DISP) {
        const int lf = f % src.nf_per_model;
        rot = src.terms[lf % src.T].w;
    }
    C *out = spec + (size_t)f * g.ncell_h;
    for (int idx = threadIdx.x; idx < n1 * per_plane_h; idx += blockDim.x) {
        const int k1 = (int)fph.div((unsigned)idx), rem = idx - k1 * per_plane_h;
        out[idx] = cipow(res3[(size_t)k1 * plane_c + rem], rot);
    }
}

// Whole field in shared memory with register-resident lines (sizes N1 x N2 x N3 known at compile
// time, every N <= 32): the field values are staged with coalesced loads as reals (rows padded to
// N3 + 1), each thread transforms two rows along axis 3 as one complex line (rows t and t + NPAIR),
// separates the two half spectra after a barrier (in place over the staged reals), then lines
// along axis 2 and axis 1 are transformed in registers; the axis-1 pass writes the half spectrum
// [k1][k2][k3 <= N3/2] straight to HBM (coalesced across the CTA), times i^n for monomials.
// One barrier per axis.
// threads per CTA: at least one per row pair of axis 3 and one per line of axes 2 and 1; more
// threads shorten the staging of the field values, which is bound by the latency of its loads
// (20³ fields: 1024 threads stage in two rounds of loads instead of four)
template <int N> constexpr int fr_threads() { return (N > 8 && N <= 20) ? 1024 : 512; }

template <typename T, int N1, int N2, int N3>
__global__ void __launch_bounds__(fr_threads<N1>(), 1) k_fft_field_reg(const Geometry g, const FieldSource src, int f0,
                                                              c_t<T> *spec) {
    using C = c_t<T>;
    constexpr int N3H = N3 / 2 + 1, NROW = N1 * N2, NPAIR = (NROW + 1) / 2, N3P = N3 + 1;
    constexpr int NCELL = N1 * N2 * N3;
    constexpr int FR_THREADS = fr_threads<N1>();
    static_assert(NPAIR <= FR_THREADS, "one row pair per thread");
    griddep_launch_dependents();   // the consumer of the spectra may be scheduled
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *buf = (C *)smem_raw;          // [N1][N2][N3H]
    T *val = (T *)smem_raw;          // staged field values [row][N3P]
    const int f = f0 + blockIdx.x, tid = threadIdx.x;
    const FieldRow<T> fr = field_row<T>(src, NCELL, f);
    // four consecutive cells per load (N3 % 4 == 0): 16-byte loads of the power rows, 4-byte loads
    // of the occupancies
    static_assert(N3 % 4 == 0, "rows of whole float4 groups");
    // values of the four cells of group c4 (cells 4 c4 .. 4 c4 + 3)
    auto load4 = [&](int c4, T (&v)[4]) {
        if (fr.kind == SRC_DISP) {
            const float4 a = ((const float4 *)fr.pw[0])[c4], b = ((const float4 *)fr.pw[1])[c4],
                         d = ((const float4 *)fr.pw[2])[c4];
            v[0] = a.x * b.x * d.x, v[1] = a.y * b.y * d.y, v[2] = a.z * b.z * d.z, v[3] = a.w * b.w * d.w;
            if (fr.occ) {
                const uchar4 o = ((const uchar4 *)fr.occ)[c4];
                v[0] *= (T)o.x, v[1] *= (T)o.y, v[2] *= (T)o.z, v[3] *= (T)o.w;
            }
        } else if (fr.kind == SRC_OCC) {
            const uchar4 o = ((const uchar4 *)fr.occ)[c4];
            v[0] = (T)o.x - fr.mean, v[1] = (T)o.y - fr.mean, v[2] = (T)o.z - fr.mean, v[3] = (T)o.w - fr.mean;
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) v[q] = row_value<T>(fr, 4 * c4 + q);
        }
    };
    auto store4 = [&](int c4, const T (&v)[4]) {
        const int c = 4 * c4, row = c / N3, r3 = c - row * N3;
#pragma unroll
        for (int q = 0; q < 4; ++q) val[row * N3P + r3 + q] = v[q];
    };
    constexpr int NG4 = NCELL / 4, NIT = (NG4 + FR_THREADS - 1) / FR_THREADS;
    if constexpr (NIT <= 2) {
        // every group of the thread loaded before any is stored: one round of load latency
        T v[NIT][4];
#pragma unroll
        for (int u = 0; u < NIT; ++u)
            if (tid + u * FR_THREADS < NG4) load4(tid + u * FR_THREADS, v[u]);
#pragma unroll
        for (int u = 0; u < NIT; ++u)
            if (tid + u * FR_THREADS < NG4) store4(tid + u * FR_THREADS, v[u]);
    } else {
        for (int c4 = tid; c4 < NG4; c4 += FR_THREADS) {
            T v[4];
            load4(c4, v);
            store4(c4, v);
        }
    }
    __syncthreads();
    // axis 3: rows t and t + NPAIR as the real and imaginary parts of one line
    C z[N3];
    const bool has1 = tid + NPAIR < NROW;
    if (tid < NPAIR) {
#pragma unroll
        for (int r3 = 0; r3 < N3; ++r3)
            z[r3] = mk<T>(val[tid * N3P + r3], has1 ? val[(tid + NPAIR) * N3P + r3] : T(0));
        RegFFT<T, N3>::run(z);
    }
    __syncthreads();
    if (tid < NPAIR) {
        // X = (Z_k + conj Z_{-k}) / 2 (row t), Y = (Z_k - conj Z_{-k}) / (2i) (row t + NPAIR)
#pragma unroll
        for (int k = 0; k < N3H; ++k) {
            const C zk = z[k], zm = z[(N3 - k) % N3];
            buf[tid * N3H + k] = mk<T>(T(0.5) * (zk.x + zm.x), T(0.5) * (zk.y - zm.y));
            if (has1) buf[(tid + NPAIR) * N3H + k] = mk<T>(T(0.5) * (zk.y + zm.y), T(-0.5) * (zk.x - zm.x));
        }
    }
    __syncthreads();
    // axis 2: line (R1, k3), elements R2 N3H apart
    for (int L = tid; L < N1 * N3H; L += FR_THREADS) {
        const int r1 = L / N3H, k3 = L - r1 * N3H;
        C *line = buf + r1 * N2 * N3H + k3;
        C y[N2];
#pragma unroll
        for (int i = 0; i < N2; ++i) y[i] = line[i * N3H];
        RegFFT<T, N2>::run(y);
#pragma unroll
        for (int i = 0; i < N2; ++i) line[i * N3H] = y[i];
    }
    __syncthreads();
    // axis 1: line (k2, k3), elements R1 N2 N3H apart; half spectrum to HBM
    int rot = 0;
    if (src.kind == SRC_DISP) rot = src.terms[(f % src.nf_per_model) % src.T].w;
    C *out = spec + (size_t)f * (N1 * N2 * N3H);
    for (int L = tid; L < N2 * N3H; L += FR_THREADS) {
        C y[N1];
#pragma unroll
        for (int i = 0; i < N1; ++i) y[i] = buf[i * N2 * N3H + L];
        RegFFT<T, N1>::run(y);
#pragma unroll
        for (int i = 0; i < N1; ++i) out[i * N2 * N3H + L] = cipow(y[i], rot);
    }
}

template <typename T, int N> static bool launch_field_reg(const Geometry &g, const FieldSource &src, int f0, int nf,
                                                          c_t<T> *spec, cudaStream_t s) {
    constexpr size_t sm = (size_t)N * N * (N / 2 + 1) * sizeof(c_t<T>);
    if (sm > 48 * 1024)
        cudaFuncSetAttribute(k_fft_field_reg<T, N, N, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_fft_field_reg<T, N, N, N><<<(unsigned)nf, fr_threads<N>(), sm, s>>>(g, src, f0, spec);
    count_launches(1);
    return true;
}

// the register kernel for cubic FP32 supercells of 8, 16, 20 or 32 cells per axis
template <typename T>
static bool fft_field_reg(const Geometry &g, const FieldSource &src, int f0, int nf, c_t<T> *spec, cudaStream_t s) {
    if constexpr (sizeof(T) != 4) {
        return false;
    } else {
        if (g.n[0] != g.n[1] || g.n[1] != g.n[2]) return false;
        switch (g.n[0]) {
            case 8: return launch_field_reg<T, 8>(g, src, f0, nf, spec, s);
            case 16: return launch_field_reg<T, 16>(g, src, f0, nf, spec, s);
            case 20: return launch_field_reg<T, 20>(g, src, f0, nf, spec, s);
            case 32: return launch_field_reg<T, 32>(g, src, f0, nf, spec, s);
            default: return false;
        }
    }
}

// ---- 64-point lines over eight threads (FP32 supercells of 64 cells per axis) -----------------
// X[k1 + 8 k2] = sum_t w64^(t k1) w8^(t k2) sum_m x[t + 8 m] w8^(m k1) (w_N = exp(+2 pi i / N)):
// thread t of a line holds x[t + 8 m], m < 8, runs the inner 8-point DFT in registers, multiplies
// by its own twiddles w64^(t k1), and the eight threads exchange values through a warp-private
// shared area so that thread k1 holds the inner results of every t; a second 8-point DFT leaves
// X[k1 + 8 k2], k2 < 8, in thread k1.  The area holds 8 rows of 9 complex per line (lines 72 apart):
// the writes and the reads of a warp each take the minimum two shared-memory wavefronts.
constexpr int F64_LS = 72, F64_RS = 9;
template <typename T>
__device__ __forceinline__ void fft64_line(c_t<T> (&v)[8], const c_t<T> (&tw)[8], c_t<T> *area, int t) {
    RegFFT<T, 8>::run(v);
#pragma unroll
    for (int k1 = 1; k1 < 8; ++k1) v[k1] = cmul(v[k1], tw[k1]);
#pragma unroll
    for (int k1 = 0; k1 < 8; ++k1) area[k1 * F64_RS + t] = v[k1];
    __syncwarp();
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = area[t * F64_RS + u];
    __syncwarp();   // the area may be written again
    RegFFT<T, 8>::run(v);
}
// the 64th roots of unity, computed by the compiler (exact octant reduction, Taylor series of the
// remainder) and rounded to FP32 once
struct Roots64 {
    float c[64], s[64];
};
constexpr Roots64 make_roots64() {
    Roots64 r{};
    for (int m = 0; m < 64; ++m) {
        r.c[m] = (float)root_cs(64, m, 0);
        r.s[m] = (float)root_cs(64, m, 1);
    }
    return r;
}
__constant__ Roots64 c_roots64 = make_roots64();
// w64^(t k1), k1 < 8
template <typename T> __device__ __forceinline__ void fft64_twiddles(int t, c_t<T> (&tw)[8]) {
#pragma unroll
    for (int k1 = 0; k1 < 8; ++k1) {
        const int m = (t * k1) & 63;
        tw[k1] = mk<T>((T)c_roots64.c[m], (T)c_roots64.s[m]);
    }
}

// Axes 3 and 2 of one 64 x 64 plane (r1 = blockIdx mod 64) of field f0 + blockIdx / 64: axis 3 on
// 32 complex lines that pack rows 2p (real) and 2p + 1 (imaginary), separated into the half spectra
// of the two rows (k3 <= 32), then axis 2 on the 33 columns; the plane [k2][k3] is written to the
// work buffer with coalesced stores.  256 threads: eight per line, four lines per warp.
template <typename T>
__global__ void __launch_bounds__(256) k_fft_planes64(const FieldSource src, int f0, c_t<T> *work) {
    using C = c_t<T>;
    constexpr int N = 64, NH = 33, PS = NH + 1;   // plane row stride (padded)
    __shared__ __align__(16) C tr[8][4][F64_LS];
    __shared__ __align__(16) C pl[N * PS];
    const int tid = threadIdx.x, warp = tid >> 5, lw = (tid >> 3) & 3, t = tid & 7;
    const int line = warp * 4 + lw;
    C *area = &tr[warp][lw][0];
    C tw[8];
    fft64_twiddles<T>(t, tw);
    const int fl = blockIdx.x >> 6, r1 = blockIdx.x & 63, f = f0 + fl;
    const FieldRow<T> fr = field_row<T>(src, N * N * N, f);
    // the plane's 64 x 64 values, staged in the plane buffer with four cells per load (rows of 68:
    // the four lines of a warp read disjoint banks)
    constexpr int SR = 68;
    static_assert(N * SR * sizeof(T) <= N * PS * sizeof(C), "staging fits the plane buffer");
    T *stage = (T *)pl;
#pragma unroll
    for (int c4 = tid; c4 < N * N / 4; c4 += 256) {
        const int cell = r1 * N * N + 4 * c4, g4 = cell >> 2;
        T x[4];
        if (fr.kind == SRC_DISP) {
            const float4 a = ((const float4 *)fr.pw[0])[g4], b = ((const float4 *)fr.pw[1])[g4],
                         d = ((const float4 *)fr.pw[2])[g4];
            x[0] = a.x * b.x * d.x, x[1] = a.y * b.y * d.y, x[2] = a.z * b.z * d.z, x[3] = a.w * b.w * d.w;
            if (fr.occ) {
                const uchar4 o = ((const uchar4 *)fr.occ)[g4];
                x[0] *= (T)o.x, x[1] *= (T)o.y, x[2] *= (T)o.z, x[3] *= (T)o.w;
            }
        } else if (fr.kind == SRC_OCC) {
            const uchar4 o = ((const uchar4 *)fr.occ)[g4];
            x[0] = (T)o.x - fr.mean, x[1] = (T)o.y - fr.mean, x[2] = (T)o.z - fr.mean, x[3] = (T)o.w - fr.mean;
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) x[q] = row_value<T>(fr, cell + q);
        }
        const int row = (4 * c4) >> 6, col = (4 * c4) & 63;
        *(float4 *)(stage + row * SR + col) = make_float4(x[0], x[1], x[2], x[3]);
    }
    __syncthreads();
    // axis 3 on the packed rows 2 line, 2 line + 1
    C v[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) v[m] = mk<T>(stage[(2 * line) * SR + t + 8 * m], stage[(2 * line + 1) * SR + t + 8 * m]);
    __syncthreads();   // the plane buffer is written below
    fft64_line<T>(v, tw, area, t);   // v[k2] = Z[t + 8 k2]
    // X = (Z_k + conj Z_-k) / 2 (row 2 line), Y = (Z_k - conj Z_-k) / (2i) (row 2 line + 1), k <= 32
#pragma unroll
    for (int k2 = 0; k2 < 8; ++k2) area[t + 8 * k2] = v[k2];
    __syncwarp();
#pragma unroll
    for (int k2 = 0; k2 < 5; ++k2) {
        const int k = t + 8 * k2;
        if (k <= 32) {
            const C zk = v[k2], zm = area[(N - k) & (N - 1)];
            pl[(2 * line) * PS + k] = mk<T>(T(0.5) * (zk.x + zm.x), T(0.5) * (zk.y - zm.y));
            pl[(2 * line + 1) * PS + k] = mk<T>(T(0.5) * (zk.y + zm.y), T(-0.5) * (zk.x - zm.x));
        }
    }
    __syncthreads();
    // axis 2 on the columns k3 (33 lines: the last one by warp 0's first eight threads)
    for (int rep = 0; rep < 2; ++rep) {
        if (rep == 1 && warp != 0) break;
        const int L = line + 32 * rep;
        const bool act = L < NH;
        C w[8];
#pragma unroll
        for (int m = 0; m < 8; ++m) w[m] = act ? pl[(t + 8 * m) * PS + L] : mk<T>(T(0), T(0));
        fft64_line<T>(w, tw, area, t);
        if (act) {
#pragma unroll
            for (int k2 = 0; k2 < 8; ++k2) pl[(t + 8 * k2) * PS + L] = w[k2];
        }
    }
    __syncthreads();
    C *out = work + (size_t)blockIdx.x * (N * NH);
#pragma unroll 4
    for (int i = tid; i < N * NH; i += 256) {
        const int k2 = i / NH, k3 = i - k2 * NH;
        out[i] = pl[k2 * PS + k3];
    }
}

// Axis 1 of 32 columns (k2, k3) of one field's work planes per block: the 64 x 32 block is staged
// in shared memory, transformed by eight threads per column, and the half spectrum written with
// coalesced rows (times i^n for Taylor monomials).  Persistent CTAs (as many as fit at once) take
// the blocks round-robin and copy the next block asynchronously into a second buffer while the
// current one is transformed, so the block loads stay in flight behind the arithmetic.
constexpr int C64_THREADS = 256;
template <typename T>
__global__ void __launch_bounds__(C64_THREADS) k_fft_columns64(const FieldSource src, int f0, int nf,
                                                               const c_t<T> *work, c_t<T> *spec) {
    using C = c_t<T>;
    constexpr int N = 64, NCOL = 64 * 33, CB = 32, CS = CB + 1, NCH = NCOL / CB;
    griddep_launch_dependents();   // the consumer of the spectra may be scheduled
    __shared__ __align__(16) C tr[8][4][F64_LS];
    extern __shared__ __align__(16) unsigned char c64_raw[];   // two blocks of N x CS values
    C(*cb)[N * CS] = (C(*)[N * CS])c64_raw;
    const int tid = threadIdx.x, warp = tid >> 5, lw = (tid >> 3) & 3, t = tid & 7;
    const int line = warp * 4 + lw;
    C *area = &tr[warp][lw][0];
    C tw[8];
    fft64_twiddles<T>(t, tw);
    const long long nblk = (long long)nf * NCH;
    // block b: field b / NCH, columns (b mod NCH) CB .. + CB - 1, 2048 values, eight copies per thread
    auto fetch = [&](long long b, int buf) {
        const int fl = (int)(b / NCH), c0 = (int)(b - (long long)fl * NCH) * CB;
        const C *in = work + (size_t)fl * N * NCOL + c0;
#pragma unroll
        for (int u = 0; u < N * CB / C64_THREADS; ++u) {
            const int i = tid + C64_THREADS * u, r = i >> 5, c = i & (CB - 1);
            cp_async<sizeof(C)>(&cb[buf][r * CS + c], in + (size_t)r * NCOL + c);
        }
        cp_async_commit();
    };
    long long b = blockIdx.x;
    if (b < nblk) fetch(b, 0);
    for (int it = 0; b < nblk; ++it, b += gridDim.x) {
        const int cur = it & 1;
        const long long bn = b + gridDim.x;
        if (bn < nblk) {
            fetch(bn, cur ^ 1);
            cp_async_wait<1>();   // this block's copies have landed (the next block's may not)
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        C *blk = cb[cur];
        C v[8];
#pragma unroll
        for (int m = 0; m < 8; ++m) v[m] = blk[(t + 8 * m) * CS + line];
        fft64_line<T>(v, tw, area, t);
#pragma unroll
        for (int k2 = 0; k2 < 8; ++k2) blk[(t + 8 * k2) * CS + line] = v[k2];
        __syncthreads();
        const int fl = (int)(b / NCH), c0 = (int)(b - (long long)fl * NCH) * CB, f = f0 + fl;
        int rot = 0;
        if (src.kind == SRC_DISP) rot = src.terms[(f % src.nf_per_model) % src.T].w;
        C *out = spec + (size_t)f * (N * NCOL) + c0;
#pragma unroll
        for (int i = tid; i < N * CB; i += C64_THREADS) {
            const int k1 = i >> 5, c = i & (CB - 1);
            out[(size_t)k1 * NCOL + c] = cipow(blk[k1 * CS + c], rot);
        }
        __syncthreads();   // the buffer is free for the copies of the block after next
    }
}

template <typename T>
static bool fft_lines64(const Geometry &g, const FieldSource &src, int f0, int nf, c_t<T> *work, c_t<T> *spec,
                        cudaStream_t s) {
    if constexpr (sizeof(T) != 4) {
        return false;
    } else {
        if (g.n[0] != 64 || g.n[1] != 64 || g.n[2] != 64 || (size_t)nf * 64 >= (1u << 31)) return false;
        k_fft_planes64<T><<<(unsigned)(nf * 64), 256, 0, s>>>(src, f0, work);
        constexpr size_t sm = 2 * 64 * 33 * sizeof(c_t<T>);   // the two block buffers
        static thread_local int c_dev = -1, c_grid = 0;
        int dev = 0;
        cudaGetDevice(&dev);
        if (dev != c_dev) {
            int nsm = 0, per = 0;
            cudaFuncSetAttribute(k_fft_columns64<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
            cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_fft_columns64<T>, C64_THREADS, sm);
            c_dev = dev, c_grid = std::max(1, nsm * std::max(per, 1));
        }
        const long long nblk = (long long)nf * 66;
        k_fft_columns64<T><<<(unsigned)std::min<long long>(nblk, c_grid), C64_THREADS, sm, s>>>(src, f0, nf, work, spec);
        count_launches(2);
        return true;
    }
}

// shared memory of the whole-field kernel (0 when a field does not fit)
static size_t field_smem(const Geometry &g, size_t ce) {
    const int n2p = (g.n[1] + 1) / 2;
    const size_t plane_c = (size_t)std::max(n2p * g.n[2], g.n[1] * g.n3h);
    const size_t b = (g.n[0] + g.n[1] + g.n[2] + 2 * (size_t)g.n[0] * plane_c) * ce;
    return b <= 150 * 1024 ? b : 0;
}

size_t fft_work_bytes(const Geometry &g, int nf, size_t elem) {
    return (size_t)nf * g.ncell_h * 2 * elem;
}

static int plane_batch(const Geometry &g, size_t celem, size_t budget) {
    const int n2p = (g.n[1] + 1) / 2;
    const size_t plane_c = (size_t)std::max(n2p * g.n[2], g.n[1] * g.n3h);
    int ppc = (int)(budget / (2 * plane_c * celem));
    ppc = std::max(1, std::min(ppc, g.n[0]));
    return ppc;
}

template <typename T>
static void fft_two_pass(const Geometry &g, const FieldSource &src, int f0, int nf, c_t<T> *work, c_t<T> *spec,
                         const c_t<T> *W1, const c_t<T> *W2, const c_t<T> *W3, cudaStream_t s) {
    using C = c_t<T>;
    const size_t ce = sizeof(C);
    // pass 1: planes per CTA bounded by 48 KB of shared memory, and small enough that the
    // grid gives a few waves over the 152 SMs even for a small batch of fields
    const int target_ctas = 152 * 4;
    int ppc = plane_batch(g, ce, 48 * 1024);
    ppc = std::max(1, std::min(ppc, (int)(((size_t)g.n[0] * nf + target_ctas - 1) / target_ctas)));
    const int n2p = (g.n[1] + 1) / 2;
    const size_t plane_c = (size_t)std::max(n2p * g.n[2], g.n[1] * g.n3h);
    size_t sm1 = (g.n[1] + g.n[2] + 2 * ppc * plane_c) * ce;
    if (sm1 > 48 * 1024) cudaFuncSetAttribute(k_fft_planes<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm1);
    dim3 g1((unsigned)(((g.n[0] + ppc - 1) / ppc) * (size_t)nf));
    k_fft_planes<T><<<g1, 256, sm1, s>>>(g, src, f0, ppc, work, W2, W3);
    // pass 2
    const int ncol = g.n[1] * g.n3h;
    int cb = (int)((48 * 1024 / ce - g.n[0]) / (2 * g.n[0]));
    cb = std::max(1, std::min(cb, ncol));
    // columns per CTA: at least 32 (coalesced rows), fewer when the batch is small
    const int cb_small = (int)(((size_t)ncol * nf + target_ctas - 1) / target_ctas);
    cb = std::max(std::min(cb, 32), std::min(cb, cb_small));
    size_t sm2 = (g.n[0] + 2 * (size_t)g.n[0] * cb) * ce;
    dim3 g2((unsigned)(((ncol + cb - 1) / cb) * (size_t)nf));
    k_fft_columns<T><<<g2, 256, sm2, s>>>(g, src, f0, cb, work, spec, W1);
    count_launches(2);
}

template <typename T>
void fft_real_fields(const Geometry &g, const FieldSource &src, int f0, int nf, c_t<T> *work, c_t<T> *spec,
                     const c_t<T> *W1, const c_t<T> *W2, const c_t<T> *W3, cudaStream_t s) {
    if (fft_field_reg<T>(g, src, f0, nf, spec, s)) return;
    if (fft_lines64<T>(g, src, f0, nf, work, spec, s)) return;
    // whole-field kernel: for batches large enough to fill the GPU with one CTA per field, on
    // supercells of at least 18^3 cells (measured on GB300: 1.4x faster than the two passes at
    // 20^3 x 1024 fields, even at 16^3 x 2000, slower for 8^3 or for fewer fields)
    if (const size_t smf = (nf >= 4 * 152 && g.ncell >= 5832) ? field_smem(g, sizeof(c_t<T>)) : 0) {
        if (smf > 48 * 1024) cudaFuncSetAttribute(k_fft_field<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smf);
        k_fft_field<T><<<(unsigned)nf, 512, smf, s>>>(g, src, f0, spec, W1, W2, W3);
        count_launches(1);
        return;
    }
    fft_two_pass<T>(g, src, f0, nf, work, spec, W1, W2, W3, s);
}

template void make_twiddles<float>(int, c_t<float> *, cudaStream_t);
template void make_twiddles<double>(int, c_t<double> *, cudaStream_t);
template void fft_real_fields<float>(const Geometry &, const FieldSource &, int, int, c_t<float> *, c_t<float> *,
                                     const c_t<float> *, const c_t<float> *, const c_t<float> *, cudaStream_t);
template void fft_real_fields<double>(const Geometry &, const FieldSource &, int, int, c_t<double> *,
                                      c_t<double> *, const c_t<double> *, const c_t<double> *,
                                      const c_t<double> *, cudaStream_t);

}  // namespace ds
