/*
 * ds.h -- C boundary of the GB300 library for FFT-based diffuse-scattering calculations
 * (J. A. M. Paddison, "Ultrafast calculation of diffuse scattering from atomistic models",
 * arXiv 1809.07088).
 *
 * A supercell model (Section II, Eq. r_def: n1 n2 n3 unit cells, nsite sites per cell) is made
 * resident in GPU memory; an intensity volume I(G) is then requested on a commensurate grid of
 * reciprocal-space points (the supercell Bragg positions of Eq. G_def), computed by the FFT
 * method of Section III (per-site transforms, Eqs. fft / comp_ft / mag_ft / U_fft / A_fft,
 * recombined by Eqs. comp_sf_diffuse / total_sf_taylor / mag_sf), with the Bragg/diffuse split
 * of Eq. bragg_diffuse_sf and optional noise reduction of Section V.
 *
 * Conventions used by every entry point:
 *  - Status codes only; no exception or longjmp crosses the boundary.  After an error,
 *    ds_last_error(ctx) returns a message (valid until the next call on that context).
 *  - The caller owns every buffer it passes.  Uploads are copied into library-owned device
 *    memory before the call returns (host sources) or in stream order (device sources).
 *  - "is_device" flags say whether a pointer is a CUDA device pointer (1) or host memory (0).
 *  - Streams are cudaStream_t passed as void* (NULL = the CUDA default stream).
 *  - Cartesian frame: a along x, b in the xy plane, c with positive z.  Spins in Bohr
 *    magnetons, displacements in Angstrom, wavevectors in 1/Angstrom including 2 pi.
 *  - Arrays are C order.  Occupancy: uint8 [model][site][n1][n2][n3] (1 = occupied).
 *    Spins and displacements: float [model][site][n1][n2][n3][3].
 *  - Intensity volumes: voxel (i, j, l) <-> Q = h0 + (i, j, l) * step, l fastest; element
 *    type double for DS_FP64, float for DS_FP32.
 *  - A context is not thread-safe, except ds_submit / ds_poll / ds_wait, which may be called
 *    from any thread.
 */
#ifndef DS_GB300_H
#define DS_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    DS_OK = 0,
    DS_ERR_ARG = -1,         /* invalid argument (message says which) */
    DS_ERR_STATE = -2,       /* call out of order, or a ticket still running (ds_poll) */
    DS_ERR_OOM = -3,         /* device allocation failed */
    DS_ERR_ADMISSION = -4,   /* request larger than the context's HBM budget */
    DS_ERR_TIMEOUT = -5,     /* a wait ran out of time (host or bounded device wait) */
    DS_ERR_CUDA = -6,        /* CUDA runtime error (message has the CUDA error string) */
    DS_ERR_UNSUPPORTED = -7  /* valid but not handled (e.g. incommensurate grid) */
} ds_status;

/* form-factor kinds (the paper leaves the functional form open, Section II / III D):
 * DS_FF_CONST   f = 1 (the scattering length b alone; neutron nuclear scattering)
 * DS_FF_GAUSS4  f(s) = sum_{i=1..4} a_i exp(-b_i s^2) + c, coef = a1 a2 a3 a4 b1 b2 b3 b4 c
 * DS_FF_J0      <j0>(s) = A exp(-a s^2) + B exp(-b s^2) + C exp(-c s^2) + D,
 *               coef = A a B b C c D (- -)
 * with s = |Q| / (4 pi). */
enum { DS_FF_CONST = 0, DS_FF_GAUSS4 = 1, DS_FF_J0 = 2 };
/* disorder type of a request: compositional (Section III B), magnetic (III D), displacive
 * (III C, Taylor expansion; carries the occupancies too when they were uploaded) */
enum { DS_OCC = 0, DS_SPIN = 1, DS_DISP = 2 };
/* DS_TOTAL: I = <|F|^2>/N (Eq. intensity_sf).  DS_DIFFUSE: I = <|F - <F>|^2>/N (Eq.
 * bragg_diffuse_sf): the occupancy deviation delta - c of Eq. occ is transformed; displacive
 * <F(H)> keeps the even Taylor orders at k = 0 (Eq. bragg_sf_disp); magnetic subtracts the
 * mean moment of each site. */
enum { DS_TOTAL = 0, DS_DIFFUSE = 1 };
/* DS_FP64: all arithmetic in double (the plain reference path).  DS_FP32: FFTs, tables and
 * recombination in float, tables generated in double. */
enum { DS_FP64 = 0, DS_FP32 = 1 };
/* noise reduction (Section V).  DS_SMOOTH_SPHERE: the Lanczos resampling with the spherically
 * symmetric cutoff W_r(|Q - G|) in place of Eq. weight_sinc (the last modification of Section
 * V B): W = W_r L, |r_c| = (1 - 1/m) |r_max| (times 2/m' for m' > 2), |r_max| the radius of the
 * sphere inscribed in the supercell; not separable, so m m' <= 16 on the grid of Bragg positions. */
enum { DS_SMOOTH_NONE = 0, DS_SMOOTH_LANCZOS = 1, DS_SMOOTH_SUBBOX = 2, DS_SMOOTH_SPHERE = 3 };

/* grid of wavevectors in r.l.u.  Only commensurate grids are handled: step = 1/n_alpha and
 * h0 * n_alpha integral (the supercell Bragg positions of Eq. G_def, Section II). */
typedef struct {
    double h0[3];
    double step[3];
    int64_t count[3];
} ds_qgrid;

typedef struct {
    int disorder;       /* DS_OCC, DS_SPIN, DS_DISP */
    int mode;           /* DS_TOTAL, DS_DIFFUSE */
    int precision;      /* DS_FP64, DS_FP32 */
    int taylor_order;   /* displacive: order P; < 0 chooses the smallest P whose remainder
                           bound x_max^(P+1)/(P+1)! <= taylor_eps (Section III C) */
    double taylor_eps;
    int smoothing;      /* DS_SMOOTH_NONE, DS_SMOOTH_LANCZOS, DS_SMOOTH_SUBBOX, DS_SMOOTH_SPHERE */
    int lanczos_m;      /* m >= 2 of Eq. lanczos */
    int lanczos_mprime; /* m' >= 2 (2 = the plain window; r_cut = (1 - 1/m)/m') */
    int subbox_n;       /* n_sb of Section V A, 1 <= n_sb <= n_alpha/2 */
    int taylor_zonal;   /* displacive with taylor_order < 0: 1 = an order per zone H of the
                           grid, from x_H = min(max_zone |Q| * max_j |u_j|, x_max), so that the
                           same remainder bound holds at every voxel (|Q.u| <= |Q||u|); 0 = one
                           order for the whole grid.  Not accepted by ds_backward. */
    int dw_coupling;    /* magnetic (DS_SPIN) only: 1 = multiply each site's term of Eq. mag_sf by
                           the Debye-Waller factor T_mu(G) of the uploaded displacements (Eq. dw,
                           even part: the mean over lattice points and supercells of cos(G.u)),
                           the only coupling of moments and displacements the paper keeps;
                           0 = T = 1.  Not with DS_SMOOTH_SUBBOX, not accepted by ds_backward. */
    int taylor_kernel;  /* displacive: how the Taylor sum of Eq. total_sf_taylor is evaluated (same sum,
                           reordered): DS_TAYLOR_AUTO picks the cheaper of the two by a cost model;
                           DS_TAYLOR_PER_VOXEL sums the monomials voxel by voxel; DS_TAYLOR_SUM_FACTORISED
                           evaluates, for every k, the polynomial in the r.l.u. coordinates over all zones
                           at once, one axis at a time (one order for the grid; DS_ERR_UNSUPPORTED when a
                           k's box of zones is wider than 17 along an axis, or with taylor_zonal). */
} ds_opts;

enum { DS_TAYLOR_AUTO = 0, DS_TAYLOR_PER_VOXEL = 1, DS_TAYLOR_SUM_FACTORISED = 2 };

typedef struct {
    int taylor_order;        /* P used (displacive), else 0 */
    int n_monomials;         /* (P+1)(P+2)(P+3)/6 */
    double x_max;            /* max |Q.u| over atoms and the requested Q box */
    double trunc_bound;      /* per-atom remainder bound x_max^(P+1)/(P+1)! */
    int64_t nvox;            /* voxels written */
    int64_t workspace_bytes; /* device scratch used by the request */
    double gpu_ms;           /* device time of the request (0 when not measured) */
    double latency_ms;       /* served requests: submit to completion (host clock), else 0 */
} ds_result_info;

typedef struct ds_ctx ds_ctx;     /* one GPU: streams, HBM budget, request queue */
typedef struct ds_model ds_model; /* one ensemble of supercells resident on that GPU */

/* Create a context on CUDA device `device`.  hbm_budget_bytes bounds the scratch a request may
 * use (0 = 90% of the free memory at creation).  Errors: DS_ERR_ARG, DS_ERR_CUDA. */
ds_status ds_create(ds_ctx **ctx, int device, size_t hbm_budget_bytes);
/* Wait for all work of the context, then free it and its models. */
ds_status ds_destroy(ds_ctx *ctx);
const char *ds_last_error(const ds_ctx *ctx);
/* Library version string. */
const char *ds_version(void);

/* Models (Section II, Eq. r_vec: r = R + r_mu + u). */
ds_status ds_model_create(ds_ctx *ctx, ds_model **model);
ds_status ds_model_destroy(ds_model *model);
/* a, b, c in Angstrom; alpha, beta, gamma in degrees. */
ds_status ds_model_set_lattice(ds_model *model, double a, double b, double c, double alpha, double beta,
                               double gamma);
/* nsite <= 64 sites at fractional coordinates frac_xyz[nsite*3]; scat_len[nsite] = b_mu
 * (NULL = 1); ff_kind[nsite] and ff_coef[nsite*9] select each site's form factor (NULL =
 * DS_FF_CONST).  Clears uploaded arrays. */
ds_status ds_model_set_sites(ds_model *model, int nsite, const double *frac_xyz, const double *scat_len,
                             const int *ff_kind, const double *ff_coef);
/* n1 n2 n3 unit cells (each 1..128 with prime factors 2, 3, 5, 7), nmodels supercells whose
 * intensities are averaged (the ensemble average of Eq. intensity_sf).  Clears arrays. */
ds_status ds_model_set_supercell(ds_model *model, int n1, int n2, int n3, int nmodels);
/* Occupancies delta (Eq. total_sf), uint8 [model][site][n1][n2][n3].  mean_occ[nsite] gives
 * c_mu of Eq. occ (NULL = sample mean over lattice points and supercells). */
ds_status ds_model_upload_occupancy(ds_model *model, const uint8_t *occ, const double *mean_occ,
                                    int src_is_device, void *stream);
/* Moments M (Eq. mag_ft), float [model][site][n1][n2][n3][3]. */
ds_status ds_model_upload_spins(ds_model *model, const float *spins, int src_is_device, void *stream);
/* Displacements u (Eq. r_vec), float [model][site][n1][n2][n3][3], Angstrom. */
ds_status ds_model_upload_displacements(ds_model *model, const float *disp, int src_is_device, void *stream);

/* I(G) on `grid` (Eqs. intensity_sf / bragg_diffuse_sf / mag_intensity and Section V), written
 * to `out` (count0*count1*count2 elements of the precision's type).  With out_is_device the
 * work is queued on `stream` and the call returns without waiting (info->gpu_ms = 0); with a
 * host `out` the call returns when the volume has been copied.  The displacive path with an
 * automatic Taylor order reads x_max back from the device first (one synchronisation).
 * Errors: DS_ERR_ARG, DS_ERR_STATE (missing arrays), DS_ERR_UNSUPPORTED (incommensurate grid,
 * unsupported size), DS_ERR_ADMISSION, DS_ERR_OOM, DS_ERR_CUDA. */
ds_status ds_request_intensity(ds_model *model, const ds_qgrid *grid, const ds_opts *opts, void *out,
                               int out_is_device, void *stream, ds_result_info *info);

/* I(Q) at npts arbitrary wavevectors (Section V B): hkl in r.l.u., [npts][3] doubles on the host
 * or (hkl_is_device) the device; out: npts values of the precision's type, host or device.  Each
 * point is resampled from I(G) on the supercell Bragg positions around it by Eq.
 * intensity_convol_finite with W = W_sinc L (Eqs. weight_sinc, windowed_sinc, lanczos;
 * opts->smoothing must be DS_SMOOTH_LANCZOS or DS_SMOOTH_SPHERE, with lanczos_m and lanczos_mprime): the sum runs
 * over floor(Q_a) - M + 1 <= G_a <= floor(Q_a) + M, M = ceil(m m'/2), inside the strict window
 * |Q_a - G_a| < m m'/2 (Q_a = n_a h_a).  I(G) is computed by the FFT method on the box of Bragg
 * positions that covers every point's support.  The points are scaled and bounded on the device;
 * the call synchronises `stream` once to read their bounds back (a few KB).  With out_is_device
 * the rest is queued on `stream` and the call returns without waiting; with a host `out` it
 * returns when the values are copied.  Errors: DS_ERR_ARG (smoothing, non-finite points), DS_ERR_ADMISSION
 * (box larger than the budget), DS_ERR_UNSUPPORTED, the errors of ds_request_intensity. */
ds_status ds_request_points(ds_model *model, const double *hkl, int64_t npts, int hkl_is_device, const ds_opts *opts,
                            void *out, int out_is_device, void *stream, ds_result_info *info);

/* Method of sub-boxes by direct summation (Section V A) at npts arbitrary wavevectors hkl
 * ([npts][3] r.l.u., host or device).  Each origin (m, o1, o2, o3) -- lattice point o of
 * supercell m -- is the corner of a box of n_sb^3 cells o + d, d in [0, n_sb)^3, with open
 * boundaries: its atoms sit at o + d + r_mu (+ u) and carry the data of the wrapped cells
 * (o + d) mod n.  I(Q) = sum_o |F_o(Q)|^2 / (norigin nsite n_sb^3) (magnetic: C |F_o,perp|^2).
 * Amplitudes: DS_OCC b delta (DIFFUSE b (delta - c_mu)); DS_SPIN b M (DIFFUSE M - <M>_mu);
 * DS_DISP b delta exp(i Q.u) with the exact exponential (delta = 1 without occupancies; DIFFUSE
 * subtracts b <delta cos(Q.u)>_mu, the Debye-Waller factor of ds_debye_waller, so that n_sb = n
 * at a supercell Bragg position gives F - <F> of Eq. bragg_sf_disp).  origins: host int32
 * [norigin][4] (the random-origin variant: origins drawn by the caller), or NULL with
 * norigin = 0 for every lattice point of every supercell.  Options read: disorder, mode,
 * precision, subbox_n (1 <= n_sb <= n_alpha; the paper keeps n_sb <= n_alpha/2 to avoid
 * periodic images).  The work is O(npts norigin nsite n_sb^3).  out: npts values of the
 * precision's type, host or device; the call synchronises `stream` before it returns.
 * Errors: DS_ERR_ARG (origins outside the supercells, non-finite points, n_sb), DS_ERR_STATE,
 * DS_ERR_UNSUPPORTED (more than 16 sites), DS_ERR_OOM, DS_ERR_ADMISSION, DS_ERR_CUDA. */
ds_status ds_request_subbox_points(ds_model *model, const int32_t *origins, int64_t norigin, const double *hkl,
                                   int64_t npts, int hkl_is_device, const ds_opts *opts, void *out, int out_is_device,
                                   void *stream, ds_result_info *info);

/* Debye-Waller factor T_mu(Q) of Eq. dw at npts wavevectors hkl ([npts][3] r.l.u., host or
 * device): out[p][mu] = mean over lattice points and supercells of w cos(Q.u_{R,mu}), the even
 * part of Eq. dw (the odd orders of Q.u average to zero over the ensemble); w = the occupancy
 * delta when occupancy_weights != 0 and occupancies are uploaded, else 1.  precision DS_FP32 or
 * DS_FP64 (type of out); synchronises `stream`.  Errors: DS_ERR_ARG, DS_ERR_STATE (no
 * displacements), DS_ERR_OOM, DS_ERR_CUDA. */
ds_status ds_debye_waller(ds_model *model, const double *hkl, int64_t npts, int hkl_is_device, int precision,
                          int occupancy_weights, void *out, int out_is_device, void *stream);

/* Serving: queue a request (device `out`, kept valid until completion).  The call validates
 * the request, chooses the Taylor order (displacive, reading x_max back on the context's own
 * stream) and estimates its HBM footprint; a worker thread admits queued requests in arrival
 * order while the footprints in flight fit the context's budget and runs each on one of eight
 * streams, so the work of concurrent requests overlaps on the GPU.  Results do not depend on
 * the mix.  The model must not be modified while its requests are in flight.  Errors:
 * DS_ERR_ADMISSION (larger than the whole budget), the errors of ds_request_intensity. */
ds_status ds_submit(ds_model *model, const ds_qgrid *grid, const ds_opts *opts, void *out, uint64_t *ticket);
/* DS_OK when finished (info filled), DS_ERR_STATE while queued or running, or the request's error. */
ds_status ds_poll(ds_ctx *ctx, uint64_t ticket, ds_result_info *info);
/* Block up to timeout_s seconds; DS_ERR_TIMEOUT if still running. */
ds_status ds_wait(ds_ctx *ctx, uint64_t ticket, double timeout_s, ds_result_info *info);

/* Hold (pause = 1) or resume (0) admission of queued requests; requests already on the GPU
 * continue.  Used to drain a context and by tests of bounded waits (no counterpart in the
 * paper). */
ds_status ds_serving_pause(ds_ctx *ctx, int pause);

/* Adjoint: given dL/dI on `grid` (same layout and type as the intensity), write dL/du
 * (displacive) or dL/dM (magnetic) in the upload layout [model][site][n1][n2][n3][3] (type of
 * the precision).  TOTAL mode, no smoothing.  The forward intensity is recomputed. */
ds_status ds_backward(ds_model *model, const ds_qgrid *grid, const ds_opts *opts, const void *dL_dI,
                      void *grad, int is_device, void *stream);

/* Tracing (no counterpart in the paper).  With profiling enabled, every kernel stage of a
 * request is bracketed by CUDA events recorded on the request stream (no synchronisation is
 * added).  ds_profile_report waits for the recorded events, then writes a JSON object
 * {"stages": {name: {"count": n, "ms": total}}, "launches": L} into json (cap bytes, NUL
 * terminated) and clears the record.  "launches" counts kernels launched by the library since
 * the previous report, whether or not profiling was enabled.  Errors: DS_ERR_ARG (buffer too
 * small), DS_ERR_CUDA. */
ds_status ds_profile_enable(ds_ctx *ctx, int enable);
ds_status ds_profile_report(ds_ctx *ctx, char *json, size_t cap);

/* Arithmetic throughput of device `device`, measured by short FMA-chain and SFU kernels (no
 * counterpart in the paper; the denominators of the ALU rooflines reported by the benchmark).  out[5]
 * (host): FP32 FMA TFLOP/s, FP32 paired FMA (float2) TFLOP/s, FP64 FMA TFLOP/s, SFU base-2
 * exponentials in 10^12 per second, SFU (sin, cos) pairs in 10^12 per second.  Synchronises the
 * device's default stream.  Errors: DS_ERR_ARG (device), DS_ERR_CUDA. */
ds_status ds_measure_peaks(int device, double out[5]);

/* Occupancy intensity for callers that cannot allocate device memory (no counterpart in the
 * paper): a host application or framework that owns all GPU memory through its own allocator,
 * a process running under a fixed memory cap, or a refinement loop that must not call the
 * allocator between iterations.  Same result as ds_request_intensity with DS_OCC, DS_FP32 and
 * constant form factors (f = 1, amplitude scat_len), computed on the CURRENT device without any
 * allocation: every intermediate lives in one static device array of 32 MiB that each GPU
 * loading the library holds until exit.
 *   lattice[6]      a, b, c (A), alpha, beta, gamma (deg);  nsite <= 32 sites at frac_xyz[nsite*3]
 *   scat_len        [nsite] host, NULL = 1;  n1 n2 n3, nmodels as for ds_model_set_supercell
 *   occ_dev         device uint8 [model][site][n1][n2][n3];  mean_occ [nsite] host or NULL
 *   grid, mode      as for ds_request_intensity (commensurate grid; DS_TOTAL / DS_DIFFUSE)
 *   out_dev         device float [count0][count1][count2], written in stream order on `stream`
 *   err, errlen     optional buffer for a message on failure
 * Requests whose scratch exceeds 32 MiB return DS_ERR_ADMISSION (message gives the size); a
 * non-finite site coordinate, scattering length or mean returns DS_ERR_ARG.  The per-site inputs
 * are passed to the GPU by value: no host buffer is read after the call returns.
 * The first call on a device (and the first after that device's context was reset) looks up the
 * array's address with that device current.  The entry point is made for direct calls on a
 * stream; recording it into a CUDA graph is not supported.  All calls share the array; calls
 * whose GPU work overlaps race on it and must be serialised by the caller.  Nothing in the array
 * needs clearing between calls. */
ds_status ds_occupancy_intensity_noalloc(const double lattice[6], int nsite, const double *frac_xyz,
                                         const double *scat_len, int n1, int n2, int n3, int nmodels,
                                         const uint8_t *occ_dev, const double *mean_occ, const ds_qgrid *grid,
                                         int mode, float *out_dev, void *stream, char *err, size_t errlen);

#ifdef __cplusplus
}
#endif

#endif /* DS_GB300_H */
