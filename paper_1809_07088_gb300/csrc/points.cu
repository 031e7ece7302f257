// Intensity at arbitrary wavevectors (Section V B): Lanczos resampling of I(G), Eq.
// intensity_convol_finite with W = W_sinc L (Eqs. weight_sinc, windowed_sinc, lanczos), for Q
// anywhere in reciprocal space (planes, lines, scattered points), not only on the grid of
// supercell Bragg positions.
//
// I(G) is computed by the FFT method on the box of Bragg positions that covers the support of
// every point (the commensurate path of api.cu), then one thread per point forms
//     I(Q) = sum_G W(Q - G) I(G) / sum_G W(Q - G)
// over floor(Q_a) - M + 1 <= G_a <= floor(Q_a) + M, M = ceil(m_eff), with the strict window
// |Q_a - G_a| < m_eff.  W is a product of one-axis weights, so are its sums; the weights are
// evaluated in FP64.  With the spherical cutoff W = W_r(|Q - G|) L(Q - G) is formed per tap.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <vector>

#include "api_internal.h"
#include "noise.h"

using namespace ds;

namespace {

constexpr double PI_D = 3.141592653589793238462643383279502884;

// one-axis weight sinc(2 pi r_cut d) sinc(pi d / m_eff) inside the window, 0 outside
__device__ __forceinline__ double axis_weight(double d, double rcut, double meff) {
    if (!(fabs(d) < meff)) return 0.0;
    if (d == 0.0) return 1.0;
    const double x1 = 2.0 * rcut * d, x2 = d / meff;  // in units of pi
    const double s1 = (x1 == 0.0) ? 1.0 : sinpi(x1) / (PI_D * x1);
    return s1 * sinpi(x2) / (PI_D * x2);
}

// MAXT: taps per axis held in registers (2M <= MAXT)
template <typename T, int MAXT>
__global__ void k_lanczos_points(const T *__restrict__ vol, int b0, int b1, int b2, int c1, int c2,
                                 const double *__restrict__ Q, long long npts, int M, double rcut, double meff,
                                 T *__restrict__ out) {
    const int ntap = 2 * M;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < npts;
         p += (long long)gridDim.x * blockDim.x) {
        double w[3][MAXT];
        double wsum[3];
        int g0[3];
        const int box[3] = {b0, b1, b2};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const double q = Q[3 * p + a];
            const double fq = floor(q);
            g0[a] = (int)fq - M + 1 - box[a];  // first tap, relative to the box origin
            wsum[a] = 0.0;
#pragma unroll
            for (int t = 0; t < MAXT; ++t) {
                double v = 0.0;
                if (t < ntap) v = axis_weight(q - (fq - M + 1 + t), rcut, meff);
                w[a][t] = v;
                wsum[a] += v;
            }
        }
        T acc = T(0);
#pragma unroll
        for (int t0 = 0; t0 < MAXT; ++t0) {
            if (t0 >= ntap || w[0][t0] == 0.0) continue;
            T acc1 = T(0);
#pragma unroll
            for (int t1 = 0; t1 < MAXT; ++t1) {
                if (t1 >= ntap || w[1][t1] == 0.0) continue;
                const T *row = vol + ((size_t)(g0[0] + t0) * c1 + (g0[1] + t1)) * c2 + g0[2];
                T acc2 = T(0);
#pragma unroll
                for (int t2 = 0; t2 < MAXT; ++t2)
                    if (t2 < ntap) acc2 = fma((T)w[2][t2], row[t2], acc2);
                acc1 = fma((T)w[1][t1], acc2, acc1);
            }
            acc = fma((T)w[0][t0], acc1, acc);
        }
        out[p] = acc / (T)(wsum[0] * wsum[1] * wsum[2]);
    }
}

// spherical cutoff: W = W_r(|Q - G|) L(Q - G) per tap (not separable), FP64 weights
struct SphereGeom {
    double qstep[9];  // a*/n1, b*/n2, c*/n3 rows: Cartesian Q - G = sum_a (Q_a - G_a) qstep_a
    double rc;        // |r_c|
};

template <typename T>
__global__ void k_sphere_points(const T *__restrict__ vol, int b0, int b1, int b2, int c1, int c2,
                                const double *__restrict__ Q, long long npts, int M, double meff,
                                const __grid_constant__ SphereGeom sg, T *__restrict__ out) {
    const int ntap = 2 * M;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < npts;
         p += (long long)gridDim.x * blockDim.x) {
        const double q[3] = {Q[3 * p], Q[3 * p + 1], Q[3 * p + 2]};
        const double fq[3] = {floor(q[0]), floor(q[1]), floor(q[2])};
        double acc = 0.0, wsum = 0.0;
        for (int t0 = 0; t0 < ntap; ++t0) {
            const double d0 = q[0] - (fq[0] - M + 1 + t0);
            if (!(fabs(d0) < meff)) continue;
            const double l0 = d0 == 0.0 ? 1.0 : sinpi(d0 / meff) / (PI_D * d0 / meff);
            for (int t1 = 0; t1 < ntap; ++t1) {
                const double d1 = q[1] - (fq[1] - M + 1 + t1);
                if (!(fabs(d1) < meff)) continue;
                const double l1 = d1 == 0.0 ? 1.0 : sinpi(d1 / meff) / (PI_D * d1 / meff);
                const T *row = vol + ((size_t)((int)fq[0] - M + 1 + t0 - b0) * c1 + ((int)fq[1] - M + 1 + t1 - b1)) * c2 +
                               ((int)fq[2] - M + 1 - b2);
                for (int t2 = 0; t2 < ntap; ++t2) {
                    const double d2 = q[2] - (fq[2] - M + 1 + t2);
                    if (!(fabs(d2) < meff)) continue;
                    const double l2 = d2 == 0.0 ? 1.0 : sinpi(d2 / meff) / (PI_D * d2 / meff);
                    double c[3];
#pragma unroll
                    for (int a = 0; a < 3; ++a) c[a] = d0 * sg.qstep[a] + d1 * sg.qstep[3 + a] + d2 * sg.qstep[6 + a];
                    const double x = sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]) * sg.rc;
                    const double wr = fabs(x) < 1e-3 ? 1.0 / 3.0 - x * x / 30.0
                                                     : sin(x) / (x * x * x) - cos(x) / (x * x);
                    const double w = wr * l0 * l1 * l2;
                    acc += w * (double)row[t2];
                    wsum += w;
                }
            }
        }
        out[p] = (T)(acc / wsum);
    }
}

template <typename T>
void launch_points(const T *vol, const int box[3], const int cnt[3], const double *dQ, long long npts, int M,
                   double rcut, double meff, T *out, cudaStream_t s) {
    const unsigned nb = (unsigned)std::max<long long>(1, std::min<long long>((npts + 127) / 128, 152 * 32));
    if (2 * M <= 4)
        k_lanczos_points<T, 4><<<nb, 128, 0, s>>>(vol, box[0], box[1], box[2], cnt[1], cnt[2], dQ, npts, M, rcut, meff, out);
    else if (2 * M <= 8)
        k_lanczos_points<T, 8><<<nb, 128, 0, s>>>(vol, box[0], box[1], box[2], cnt[1], cnt[2], dQ, npts, M, rcut, meff, out);
    else if (2 * M <= 16)
        k_lanczos_points<T, 16><<<nb, 128, 0, s>>>(vol, box[0], box[1], box[2], cnt[1], cnt[2], dQ, npts, M, rcut, meff, out);
    else
        k_lanczos_points<T, 64><<<nb, 128, 0, s>>>(vol, box[0], box[1], box[2], cnt[1], cnt[2], dQ, npts, M, rcut, meff, out);
    count_launches(1);
}

// Q_a = n_a h_a (supercell-index units) written to Q, and per block the range of floor(Q_a) over
// the finite points and the index of the first non-finite one (slots lo[3], hi[3], bad).  hkl and
// Q may be the same buffer: each element is read and written by one thread.
constexpr int PB_THREADS = 256;
constexpr int PB_SLOTS = 7;

__global__ void __launch_bounds__(PB_THREADS)
    k_points_scale(const double *hkl, long long npts, double n0, double n1, double n2, double *Q, double *part) {
    const double n[3] = {n0, n1, n2};
    double v[PB_SLOTS] = {INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY, INFINITY};
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < npts;
         p += (long long)gridDim.x * blockDim.x) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const double q = hkl[3 * p + a] * n[a];
            Q[3 * p + a] = q;
            if (!isfinite(q)) {
                v[6] = fmin(v[6], (double)p);
            } else {
                const double f = floor(q);
                v[a] = fmin(v[a], f);
                v[3 + a] = fmax(v[3 + a], f);
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int s = 0; s < PB_SLOTS; ++s) {
            const double w = __shfl_xor_sync(0xffffffffu, v[s], o);
            v[s] = (s >= 3 && s < 6) ? fmax(v[s], w) : fmin(v[s], w);
        }
    __shared__ double red[PB_THREADS / 32][PB_SLOTS];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0)
#pragma unroll
        for (int s = 0; s < PB_SLOTS; ++s) red[wid][s] = v[s];
    __syncthreads();
    if (threadIdx.x < PB_SLOTS) {
        const int s = threadIdx.x;
        double r = red[0][s];
        for (int w = 1; w < PB_THREADS / 32; ++w) r = (s >= 3 && s < 6) ? fmax(r, red[w][s]) : fmin(r, red[w][s]);
        part[(size_t)blockIdx.x * PB_SLOTS + s] = r;
    }
}

// dQ: the points in supercell-index units on the device; fl_lo/fl_hi: the range of floor(Q_a)
template <typename T>
ds_status run_points(ds_model *Mdl, const double *dQ, const double fl_lo[3], const double fl_hi[3], long long npts,
                     const ds_opts *o, void *out, int out_dev, cudaStream_t st, Scratch &ws, ds_result_info *info) {
    ds_ctx *ctx = Mdl->ctx;
    const int m = o->lanczos_m, mp = o->lanczos_mprime;
    const double rcut = (1.0 - 1.0 / m) / mp, meff = 0.5 * m * mp;
    const int M = (int)std::ceil(meff);
    // box of Bragg positions covering every point's support: floor(Q_a) - M + 1 .. floor(Q_a) + M
    ds_qgrid box;
    int b[3], cnt[3];
    size_t nvox = 1;
    for (int a = 0; a < 3; ++a) {
        if (!(std::fabs(fl_lo[a]) <= 1e8 && std::fabs(fl_hi[a]) <= 1e8) || fl_hi[a] - fl_lo[a] + 2 * M > (1 << 20))
            return ds_fail(ctx, DS_ERR_UNSUPPORTED, "points span too many Bragg positions along axis %d", a);
        b[a] = (int)fl_lo[a] - M + 1;
        cnt[a] = (int)(fl_hi[a] - fl_lo[a]) + 2 * M;
        box.h0[a] = (double)b[a] / Mdl->n[a];
        box.step[a] = 1.0 / Mdl->n[a];
        box.count[a] = cnt[a];
        nvox *= (size_t)cnt[a];
    }
    if (nvox * sizeof(T) > ctx->budget)
        return ds_fail(ctx, DS_ERR_ADMISSION, "the box of Bragg positions under the points needs %zu bytes, budget %zu",
                       nvox * sizeof(T), ctx->budget);
    ds_opts ob = *o;
    ob.smoothing = DS_SMOOTH_NONE;
    T *vol = (T *)ws.get(sizeof(T) * nvox);
    T *dout = out_dev ? (T *)out : (T *)ws.get(sizeof(T) * npts);
    if (ws.failed) return ds_fail(ctx, DS_ERR_OOM, "device allocation failed (points)");
    ds_status rc = plan_and_run<T>(Mdl, &box, &ob, vol, st, ws, info, nullptr);
    if (rc != DS_OK) return rc;
    if (o->smoothing == DS_SMOOTH_SPHERE) {
        ProfScope ps(ctx, "lanczos_points", st);
        SphereGeom sg;
        for (int i = 0; i < 9; ++i) sg.qstep[i] = Mdl->recip[i] / Mdl->n[i / 3];
        sg.rc = sphere_cutoff_radius(Mdl, m, mp);
        const unsigned nb = (unsigned)std::max<long long>(1, std::min<long long>((npts + 127) / 128, 152 * 32));
        k_sphere_points<T><<<nb, 128, 0, st>>>(vol, b[0], b[1], b[2], cnt[1], cnt[2], dQ, npts, M, meff, sg, dout);
        count_launches(1);
    } else {
        ProfScope ps(ctx, "lanczos_points", st);
        launch_points<T>(vol, b, cnt, dQ, npts, M, rcut, meff, dout, st);
    }
    if (cudaGetLastError() != cudaSuccess) return ds_fail(ctx, DS_ERR_CUDA, "points launch failed");
    if (!out_dev && cudaMemcpyAsync(out, dout, sizeof(T) * npts, cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return ds_fail(ctx, DS_ERR_CUDA, "copy of the intensities to the host failed");
    ws.release();
    // a host output is complete on return; a device output is ordered on the stream
    if (!out_dev && cudaStreamSynchronize(st) != cudaSuccess)
        return ds_fail(ctx, DS_ERR_CUDA, "stream synchronisation failed: %s", cudaGetErrorString(cudaGetLastError()));
    if (info) info->nvox = npts;
    return DS_OK;
}

}  // namespace

extern "C" ds_status ds_request_points(ds_model *Mdl, const double *hkl, int64_t npts, int hkl_is_device,
                                       const ds_opts *o, void *out, int out_is_device, void *stream,
                                       ds_result_info *info) {
    if (!Mdl) return DS_ERR_ARG;
    ds_ctx *ctx = Mdl->ctx;
    if (!o) return ds_fail(ctx, DS_ERR_ARG, "null options");
    if (npts < 0) return ds_fail(ctx, DS_ERR_ARG, "negative point count");
    if (npts > 0 && (!hkl || !out)) return ds_fail(ctx, DS_ERR_ARG, "null points or output");
    if (o->smoothing != DS_SMOOTH_LANCZOS && o->smoothing != DS_SMOOTH_SPHERE)
        return ds_fail(ctx, DS_ERR_ARG, "points off the Bragg grid need smoothing = DS_SMOOTH_LANCZOS or DS_SMOOTH_SPHERE");
    if (!Mdl->has_cells) return ds_fail(ctx, DS_ERR_STATE, "model incomplete");
    if (info) memset(info, 0, sizeof(*info));
    if (npts == 0) return DS_OK;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return ds_fail(ctx, DS_ERR_CUDA, "cudaSetDevice");
    cudaStream_t st = (cudaStream_t)stream;
    // options and model state, checked on a one-voxel grid at the origin before any work is queued
    ds_qgrid probe;
    for (int a = 0; a < 3; ++a) {
        probe.h0[a] = 0.0;
        probe.step[a] = 1.0 / Mdl->n[a];
        probe.count[a] = 1;
    }
    ds_status rc = check_request(Mdl, &probe, o);
    if (rc != DS_OK) return rc;
    // the points scaled to Q_a = n_a h_a on the device; only their per-block bounds come back
    Scratch ws(st);
    const unsigned nb = (unsigned)std::max<long long>(1, std::min<long long>((npts + PB_THREADS - 1) / PB_THREADS, 152 * 2));
    double *dQ = (double *)ws.get(sizeof(double) * 3 * npts);
    double *dpart = (double *)ws.get(sizeof(double) * PB_SLOTS * nb);
    if (ws.failed) return ds_fail(ctx, DS_ERR_OOM, "device allocation failed (points)");
    if (!hkl_is_device && cudaMemcpyAsync(dQ, hkl, sizeof(double) * 3 * npts, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return ds_fail(ctx, DS_ERR_CUDA, "copy of the points failed");
    k_points_scale<<<nb, PB_THREADS, 0, st>>>(hkl_is_device ? hkl : dQ, npts, (double)Mdl->n[0], (double)Mdl->n[1],
                                             (double)Mdl->n[2], dQ, dpart);
    count_launches(1);
    if (cudaGetLastError() != cudaSuccess) return ds_fail(ctx, DS_ERR_CUDA, "points launch failed");
    std::vector<double> part((size_t)PB_SLOTS * nb);
    if (cudaMemcpyAsync(part.data(), dpart, sizeof(double) * part.size(), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return ds_fail(ctx, DS_ERR_CUDA, "read-back of the point bounds failed: %s", cudaGetErrorString(cudaGetLastError()));
    double lo[3], hi[3], bad = INFINITY;
    for (int a = 0; a < 3; ++a) {
        lo[a] = INFINITY;
        hi[a] = -INFINITY;
    }
    for (unsigned k = 0; k < nb; ++k) {
        const double *v = part.data() + (size_t)k * PB_SLOTS;
        for (int a = 0; a < 3; ++a) {
            lo[a] = std::min(lo[a], v[a]);
            hi[a] = std::max(hi[a], v[3 + a]);
        }
        bad = std::min(bad, v[6]);
    }
    if (bad < INFINITY) return ds_fail(ctx, DS_ERR_ARG, "point %lld is not finite", (long long)bad);
    if (o->precision == DS_FP64) return run_points<double>(Mdl, dQ, lo, hi, npts, o, out, out_is_device, st, ws, info);
    return run_points<float>(Mdl, dQ, lo, hi, npts, o, out, out_is_device, st, ws, info);
}
