// C-ABI runtime: contexts, resident supercell models, request planning and the launch sequence
// of the FFT method (Section III) with the noise-reduction step (Section V).
//
// Planning happens on the host in FP64 (grid validation, zone ranges, Taylor order, the
// monomial list); every step of the calculation itself runs in the kernels of fft.cu,
// recomb.cu, noise.cu, subbox.cu and adjoint.cu.  Request scratch comes from the device's
// stream-ordered memory pool (cudaMallocAsync / cudaFreeAsync on the request stream), so
// repeated requests reuse the same memory without synchronising.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/ds.h"
#include "api_internal.h"
#include "internal.h"
#include "noise.h"

using namespace ds;

// ------------------------------------------------------------------------------------------
// errors
// ------------------------------------------------------------------------------------------

ds_status ds_fail(ds_ctx *ctx, ds_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (ctx) {
        std::lock_guard<std::mutex> g(ctx->err_mu);
        ctx->err = buf;
    }
    return st;
}

#define CK(call)                                                                                  \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess) return ds_fail(ctx, DS_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

// ------------------------------------------------------------------------------------------
// geometry helpers (host, FP64)
// ------------------------------------------------------------------------------------------

void lattice_matrices(const double lat[6], double A[9], double B[9]) {
    const double d2r = 3.14159265358979323846 / 180.0;
    const double a = lat[0], b = lat[1], c = lat[2];
    const double al = lat[3] * d2r, be = lat[4] * d2r, ga = lat[5] * d2r;
    const double cx = c * cos(be);
    const double cy = c * (cos(al) - cos(be) * cos(ga)) / sin(ga);
    const double cz = sqrt(std::max(0.0, c * c - cx * cx - cy * cy));
    const double Am[9] = {a, 0, 0, b * cos(ga), b * sin(ga), 0, cx, cy, cz};
    memcpy(A, Am, sizeof(Am));
    // B rows = 2 pi (A^-1)^T rows: b_i* . a_j = 2 pi delta_ij
    const double det = Am[0] * (Am[4] * Am[8] - Am[5] * Am[7]) - Am[1] * (Am[3] * Am[8] - Am[5] * Am[6]) +
                       Am[2] * (Am[3] * Am[7] - Am[4] * Am[6]);
    double inv[9];
    inv[0] = (Am[4] * Am[8] - Am[5] * Am[7]) / det;
    inv[1] = (Am[2] * Am[7] - Am[1] * Am[8]) / det;
    inv[2] = (Am[1] * Am[5] - Am[2] * Am[4]) / det;
    inv[3] = (Am[5] * Am[6] - Am[3] * Am[8]) / det;
    inv[4] = (Am[0] * Am[8] - Am[2] * Am[6]) / det;
    inv[5] = (Am[2] * Am[3] - Am[0] * Am[5]) / det;
    inv[6] = (Am[3] * Am[7] - Am[4] * Am[6]) / det;
    inv[7] = (Am[1] * Am[6] - Am[0] * Am[7]) / det;
    inv[8] = (Am[0] * Am[4] - Am[1] * Am[3]) / det;
    const double two_pi = 6.283185307179586476925286766559;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) B[3 * i + j] = two_pi * inv[3 * j + i];
}

// order the stream after an event, unless the event's work has already completed (then the wait
// is a no-op; skipping it also keeps a request capturable into a CUDA graph when the event was
// recorded before the capture began)
static cudaError_t wait_unless_done(cudaStream_t st, cudaEvent_t ev) {
    const cudaError_t q = cudaEventQuery(ev);
    if (q == cudaSuccess) return cudaSuccess;
    if (q != cudaErrorNotReady) return q;
    return cudaStreamWaitEvent(st, ev, 0);
}

static bool plan_axis(int n, AxisPlan &p) {
    p.n = n;
    p.nrad = 0;
    int m = n;
    const int order[5] = {4, 2, 3, 5, 7};
    for (int r : order) {
        while (m % r == 0) {
            if (p.nrad == 8) return false;
            p.rad[p.nrad++] = r;
            m /= r;
        }
    }
    int Ns = 1;
    for (int q = 0; q < p.nrad; ++q) {
        p.mNR[q] = FastDiv::magic((unsigned)(n / p.rad[q]));
        p.mNs[q] = FastDiv::magic((unsigned)Ns);
        Ns *= p.rad[q];
    }
    return m == 1;
}

bool make_geometry(const int n[3], Geometry &g) {
    for (int a = 0; a < 3; ++a) {
        g.n[a] = n[a];
        if (n[a] < 1 || n[a] > 128 || !plan_axis(n[a], g.ax[a])) return false;
    }
    g.n3h = n[2] / 2 + 1;
    g.ncell = n[0] * n[1] * n[2];
    g.ncell_h = n[0] * n[1] * g.n3h;
    return true;
}

static int64_t floor_div64(int64_t a, int64_t b) {
    int64_t q = a / b;
    if ((a % b != 0) && ((a < 0) != (b < 0))) --q;
    return q;
}

// validate a commensurate grid; g0/cnt in supercell indices
ds_status grid_indices(ds_ctx *ctx, const ds_model *M, const ds_qgrid *q, int g0[3], int cnt[3]) {
    for (int a = 0; a < 3; ++a) {
        const double n = M->n[a];
        if (q->count[a] < 1 || q->count[a] > (1 << 20)) return ds_fail(ctx, DS_ERR_ARG, "grid count[%d] out of range", a);
        const double s = q->step[a] * n;
        if (!(fabs(s - 1.0) < 1e-9)) {
            return ds_fail(ctx, DS_ERR_UNSUPPORTED,
                           "grid axis %d: step %.17g is not 1/n (only commensurate grids of supercell "
                           "Bragg positions are handled)", a, q->step[a]);
        }
        const double x = q->h0[a] * n;
        const double r = std::nearbyint(x);
        if (!(fabs(x - r) < 1e-6)) return ds_fail(ctx, DS_ERR_UNSUPPORTED, "grid axis %d: h0 * n is not integral", a);
        if (fabs(r) > 1e8) return ds_fail(ctx, DS_ERR_ARG, "grid axis %d: h0 too large", a);
        g0[a] = (int)r;
        cnt[a] = (int)q->count[a];
    }
    return DS_OK;
}

GridMap grid_map(const Geometry &g, const int g0[3], const int cnt[3]) {
    GridMap gm;
    for (int a = 0; a < 3; ++a) {
        gm.g0[a] = g0[a];
        gm.cnt[a] = cnt[a];
        gm.Hmin[a] = (int)floor_div64(g0[a], g.n[a]);
        const int Hmax = (int)floor_div64((int64_t)g0[a] + cnt[a] - 1, g.n[a]);
        gm.nH[a] = Hmax - gm.Hmin[a] + 1;
    }
    return gm;
}

// monomials (a, b, c) with a + b + c <= P in lexicographic order, and the coefficient update
// code of each (see the displacive recombination kernel)
void monomial_tables(int P, std::vector<int4> &terms, std::vector<int> &ops) {
    terms.clear();
    ops.clear();
    for (int a = 0; a <= P; ++a)
        for (int b = 0; b <= P - a; ++b)
            for (int c = 0; c <= P - a - b; ++c) {
                terms.push_back(make_int4(a, b, c, a + b + c));
                int op;
                if (a == 0 && b == 0 && c == 0) op = 3;
                else if (c > 0) op = 0;
                else if (b > 0) op = 1;
                else op = 2;
                ops.push_back(op);
            }
}

int taylor_order_for(double xmax, double eps) {
    int P = 0;
    const double le = log(eps);
    while ((P + 1) * log(std::max(xmax, 1e-300)) - lgamma((double)P + 2.0) > le) {
        ++P;
        if (P > 200) return -1;
    }
    return P;
}

// sites sorted into form-factor classes (contiguous ranges)
template <typename T>
static bool form_factor_classes(const ds_model *M, std::vector<int> &site_of, FormFactors<T> &ff) {
    const int ns = M->nsite;
    site_of.resize(ns);
    for (int i = 0; i < ns; ++i) site_of[i] = i;
    auto key_less = [&](int x, int y) {
        const int kx = M->ffkind[x], ky = M->ffkind[y];
        if (kx != ky) return kx < ky;
        if (kx == DS_FF_CONST) return false;
        for (int j = 0; j < 9; ++j)
            if (M->ffcoef[9 * x + j] != M->ffcoef[9 * y + j]) return M->ffcoef[9 * x + j] < M->ffcoef[9 * y + j];
        return false;
    };
    std::stable_sort(site_of.begin(), site_of.end(), key_less);
    // within a class, order by z = r3 mod 1 so that sites sharing exp(2 pi i H3 z) are adjacent
    auto zfrac = [&](int s) { double z = M->sites[3 * s + 2]; return z - floor(z); };
    for (int i = 0; i < ns;) {
        int j = i + 1;
        while (j < ns && !key_less(site_of[i], site_of[j]) && !key_less(site_of[j], site_of[i])) ++j;
        std::stable_sort(site_of.begin() + i, site_of.begin() + j, [&](int x, int y) { return zfrac(x) < zfrac(y); });
        i = j;
    }
    ff.ncls = 0;
    for (int i = 0; i < ns; ++i) {
        const bool same = i > 0 && !key_less(site_of[i - 1], site_of[i]) && !key_less(site_of[i], site_of[i - 1]);
        if (!same) {
            if (ff.ncls == MAX_FF_CLASSES) return false;
            const int s = site_of[i];
            ff.cls_kind[ff.ncls] = M->ffkind[s];
            for (int j = 0; j < 9; ++j) ff.cls_coef[ff.ncls][j] = (T)M->ffcoef[9 * s + j];
            gaussian_sum_form(ff, ff.ncls, M->ffkind[s], &M->ffcoef[9 * s]);
            ff.ncls++;
        }
        ff.cls_end[ff.ncls - 1] = i + 1;
    }
    for (int c = ff.ncls; c < MAX_FF_CLASSES; ++c) ff.cls_end[c] = -1;
    return true;
}

// ------------------------------------------------------------------------------------------
// stream-ordered scratch
// ------------------------------------------------------------------------------------------

Scratch::~Scratch() { release(); }
void *Scratch::get(size_t bytes) {
    if (bytes == 0) bytes = 16;
    void *p = nullptr;
    cudaError_t e = cudaMallocAsync(&p, bytes, stream);
    if (e != cudaSuccess) {
        failed = true;
        cudaGetLastError();
        return nullptr;
    }
    ptrs.push_back(p);
    total += bytes;
    return p;
}
void Scratch::release() {
    for (void *p : ptrs) cudaFreeAsync(p, stream);
    ptrs.clear();
}

// ------------------------------------------------------------------------------------------
// context and models
// ------------------------------------------------------------------------------------------

extern "C" const char *ds_version(void) { return "paper_1809_07088_gb300 0.1 (sm_103a)"; }

extern "C" ds_status ds_create(ds_ctx **out, int device, size_t budget) {
    if (!out) return DS_ERR_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return DS_ERR_ARG;
    }
    if (cudaSetDevice(device) != cudaSuccess) return DS_ERR_CUDA;
    ds_ctx *ctx = new ds_ctx();
    ctx->device = device;
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    ctx->budget = budget ? budget : (size_t)(0.9 * (double)fr);
    if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete ctx;
        return DS_ERR_CUDA;
    }
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    cudaGetLastError();
    *out = ctx;
    return DS_OK;
}

extern "C" ds_status ds_destroy(ds_ctx *ctx) {
    if (!ctx) return DS_ERR_ARG;
    serving_shutdown(ctx);
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    for (ds_model *m : std::vector<ds_model *>(ctx->models.begin(), ctx->models.end())) ds_model_destroy(m);
    for (auto &r : ctx->prof) {
        cudaEventDestroy(r.e0);
        cudaEventDestroy(r.e1);
    }
    for (cudaEvent_t e : ctx->event_pool) cudaEventDestroy(e);
    cudaStreamDestroy(ctx->stream);
    delete ctx;
    return DS_OK;
}

extern "C" const char *ds_last_error(const ds_ctx *ctx) {
    if (!ctx) return "null context";
    return ctx->err.c_str();
}

extern "C" ds_status ds_model_create(ds_ctx *ctx, ds_model **out) {
    if (!ctx || !out) return ds_fail(ctx, DS_ERR_ARG, "null argument");
    ds_model *m = new ds_model();
    m->ctx = ctx;
    ctx->models.insert(m);
    *out = m;
    return DS_OK;
}

static void clear_site_tables(ds_model *m) {
    for (auto &kv : m->site_tables) {
        cudaFree(kv.second.phk);
        cudaFree(kv.second.phH);
        cudaEventDestroy(kv.second.done);
    }
    m->site_tables.clear();
}

static void free_arrays(ds_model *m) {
    cudaSetDevice(m->ctx->device);
    cudaDeviceSynchronize();
    for (void *p : {(void *)m->d_occ, (void *)m->d_spins, (void *)m->d_disp, (void *)m->d_mean_occ,
                    (void *)m->d_mean_spin})
        if (p) cudaFree(p);
    m->d_occ = nullptr;
    m->d_spins = nullptr;
    m->d_disp = nullptr;
    m->d_mean_occ = nullptr;
    m->d_mean_spin = nullptr;
    clear_site_tables(m);
}

static void free_constants(ds_model *m) {
    cudaSetDevice(m->ctx->device);
    cudaDeviceSynchronize();
    for (void *p : {(void *)m->d_site_of, (void *)m->d_scat32, (void *)m->d_scat64, (void *)m->d_user_mean})
        if (p) cudaFree(p);
    m->d_site_of = nullptr;
    m->d_scat32 = nullptr;
    m->d_scat64 = nullptr;
    m->d_user_mean = nullptr;
    for (auto &kv : m->taylor_tables) {
        cudaFree(kv.second.first);
        cudaFree(kv.second.second);
    }
    m->taylor_tables.clear();
    for (auto &kv : m->sub_tables) cudaFree(kv.second);
    m->sub_tables.clear();
    clear_site_tables(m);
}

static void free_twiddles(ds_model *m) {
    for (int a = 0; a < 3; ++a) {
        if (m->d_tw32[a]) cudaFree(m->d_tw32[a]);
        if (m->d_tw64[a]) cudaFree(m->d_tw64[a]);
        m->d_tw32[a] = nullptr;
        m->d_tw64[a] = nullptr;
    }
}

extern "C" ds_status ds_model_destroy(ds_model *m) {
    if (!m) return DS_ERR_ARG;
    free_arrays(m);
    free_constants(m);
    free_twiddles(m);
    if (m->ready) cudaEventDestroy(m->ready);
    if (m->d_sites) cudaFree(m->d_sites);
    m->ctx->models.erase(m);
    delete m;
    return DS_OK;
}

extern "C" ds_status ds_model_set_lattice(ds_model *m, double a, double b, double c, double al, double be,
                                          double ga) {
    if (!m) return DS_ERR_ARG;
    ds_ctx *ctx = m->ctx;
    if (!(a > 0 && b > 0 && c > 0) || !(al > 0 && al < 180 && be > 0 && be < 180 && ga > 0 && ga < 180))
        return ds_fail(ctx, DS_ERR_ARG, "invalid lattice parameters");
    const double lat[6] = {a, b, c, al, be, ga};
    double A[9], B[9];
    lattice_matrices(lat, A, B);
    if (!(A[8] > 0) || !std::isfinite(B[0])) return ds_fail(ctx, DS_ERR_ARG, "degenerate lattice");
    memcpy(m->lat, lat, sizeof(lat));
    memcpy(m->A, A, sizeof(A));
    memcpy(m->recip, B, sizeof(B));
    m->has_lattice = true;
    return DS_OK;
}

extern "C" ds_status ds_model_set_sites(ds_model *m, int nsite, const double *xyz, const double *scat,
                                        const int *kind, const double *coef) {
    if (!m) return DS_ERR_ARG;
    ds_ctx *ctx = m->ctx;
    if (nsite < 1 || nsite > MAX_SITES || !xyz) return ds_fail(ctx, DS_ERR_ARG, "nsite must be 1..%d", MAX_SITES);
    for (int i = 0; i < nsite; ++i) {
        if (kind && (kind[i] < 0 || kind[i] > 2)) return ds_fail(ctx, DS_ERR_ARG, "form-factor kind of site %d", i);
        for (int a = 0; a < 3; ++a)
            if (!std::isfinite(xyz[3 * i + a])) return ds_fail(ctx, DS_ERR_ARG, "site %d coordinate", i);
    }
    free_arrays(m);
    m->has_occ = m->has_spins = m->has_disp = false;
    m->nsite = nsite;
    m->sites.assign(xyz, xyz + 3 * nsite);
    m->scat.assign(nsite, 1.0);
    if (scat) m->scat.assign(scat, scat + nsite);
    m->ffkind.assign(nsite, DS_FF_CONST);
    if (kind) m->ffkind.assign(kind, kind + nsite);
    m->ffcoef.assign(9 * nsite, 0.0);
    if (coef) m->ffcoef.assign(coef, coef + 9 * nsite);
    cudaSetDevice(ctx->device);
    if (m->d_sites) cudaFree(m->d_sites);
    m->d_sites = nullptr;
    free_constants(m);
    CK(cudaMalloc(&m->d_sites, sizeof(double) * 3 * nsite));
    CK(cudaMemcpy(m->d_sites, xyz, sizeof(double) * 3 * nsite, cudaMemcpyHostToDevice));
    m->ff_ok = form_factor_classes<float>(m, m->site_of, m->ff32) && form_factor_classes<double>(m, m->site_of, m->ff64);
    if (m->ff_ok) {
        // groups: consecutive sorted sites of one class with equal z mod 1
        SiteGroups &G = m->groups;
        memset(&G, 0, sizeof(G));
        int cls = 0;
        double zprev = -1.0;
        for (int i = 0; i < nsite; ++i) {
            bool boundary = i == 0;
            if (i > 0 && i == m->ff64.cls_end[cls]) {
                G.cls_grp_end[cls] = G.ngrp;
                ++cls;
                boundary = true;
            }
            const int s = m->site_of[i];
            const double z = m->sites[3 * s + 2] - floor(m->sites[3 * s + 2]);
            if (boundary || z != zprev) {
                G.grp_site[G.ngrp] = s;
                G.ngrp++;
            }
            G.grp_end[G.ngrp - 1] = i + 1;
            zprev = z;
        }
        G.cls_grp_end[cls] = G.ngrp;
        for (int c = cls + 1; c < MAX_FF_CLASSES; ++c) G.cls_grp_end[c] = -1;
    }
    // periods of the zone phases exp(2 pi i H_a r_mu,a): every coordinate a multiple of 1/d
    for (int a = 0; a < 3; ++a) {
        m->period[a] = 0;
        for (int d = 1; d <= 64 && !m->period[a]; ++d) {
            bool ok = true;
            for (int i = 0; i < nsite && ok; ++i) {
                const double x = d * m->sites[3 * i + a];
                ok = fabs(x - rint(x)) <= 1e-13;
            }
            if (ok) m->period[a] = d;
        }
    }
    std::vector<float> s32(nsite);
    for (int i = 0; i < nsite; ++i) s32[i] = (float)m->scat[i];
    CK(cudaMalloc(&m->d_site_of, sizeof(int) * nsite));
    CK(cudaMalloc(&m->d_scat32, sizeof(float) * nsite));
    CK(cudaMalloc(&m->d_scat64, sizeof(double) * nsite));
    CK(cudaMemcpy(m->d_site_of, m->site_of.data(), sizeof(int) * nsite, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(m->d_scat32, s32.data(), sizeof(float) * nsite, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(m->d_scat64, m->scat.data(), sizeof(double) * nsite, cudaMemcpyHostToDevice));
    return DS_OK;
}

// for every order p <= P, the lexicographic monomials of order <= p as indices into the order-P
// list, with their coefficient update codes: [map | ops | off[P+2]] on the device, per model
static ds_status sub_simplex_tables(ds_model *m, int P, int **tab) {
    ds_ctx *ctx = m->ctx;
    // the serving worker and caller threads plan requests on the same model concurrently
    std::lock_guard<std::mutex> lk(m->cache_mu);
    auto it = m->sub_tables.find(P);
    if (it != m->sub_tables.end()) {
        *tab = it->second;
        return DS_OK;
    }
    std::vector<int4> terms;
    std::vector<int> ops;
    monomial_tables(P, terms, ops);
    std::map<long long, int> index;
    for (size_t t = 0; t < terms.size(); ++t)
        index[((long long)terms[t].x * 1024 + terms[t].y) * 1024 + terms[t].z] = (int)t;
    std::vector<int> map, sops, off;
    for (int p = 0; p <= P; ++p) {
        off.push_back((int)map.size());
        std::vector<int4> tp;
        std::vector<int> op;
        monomial_tables(p, tp, op);
        for (size_t t = 0; t < tp.size(); ++t) {
            map.push_back(index[((long long)tp[t].x * 1024 + tp[t].y) * 1024 + tp[t].z]);
            sops.push_back(op[t]);
        }
    }
    off.push_back((int)map.size());
    const size_t n = map.size();
    std::vector<int> all(2 * n + off.size());
    std::copy(map.begin(), map.end(), all.begin());
    std::copy(sops.begin(), sops.end(), all.begin() + n);
    for (size_t i = 0; i < off.size(); ++i) all[2 * n + i] = off[i];
    int *d = nullptr;
    CK(cudaMalloc(&d, sizeof(int) * all.size()));
    CK(cudaMemcpy(d, all.data(), sizeof(int) * all.size(), cudaMemcpyHostToDevice));
    m->sub_tables[P] = d;
    *tab = d;
    return DS_OK;
}

// monomial tables of order P on the device, built once per model and order
static ds_status taylor_tables(ds_model *m, int P, int4 **terms, int **ops, int *T) {
    ds_ctx *ctx = m->ctx;
    std::vector<int4> t;
    std::vector<int> o;
    monomial_tables(P, t, o);
    *T = (int)t.size();
    std::lock_guard<std::mutex> lk(m->cache_mu);
    auto it = m->taylor_tables.find(P);
    if (it == m->taylor_tables.end()) {
        int4 *dt = nullptr;
        int *dop = nullptr;
        CK(cudaMalloc(&dt, sizeof(int4) * t.size()));
        CK(cudaMalloc(&dop, sizeof(int) * o.size()));
        CK(cudaMemcpy(dt, t.data(), sizeof(int4) * t.size(), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(dop, o.data(), sizeof(int) * o.size(), cudaMemcpyHostToDevice));
        it = m->taylor_tables.emplace(P, std::make_pair(dt, dop)).first;
    }
    *terms = it->second.first;
    *ops = it->second.second;
    return DS_OK;
}

extern "C" ds_status ds_model_set_supercell(ds_model *m, int n1, int n2, int n3, int nmodels) {
    if (!m) return DS_ERR_ARG;
    ds_ctx *ctx = m->ctx;
    const int n[3] = {n1, n2, n3};
    Geometry g;
    if (nmodels < 1 || nmodels > 100000) return ds_fail(ctx, DS_ERR_ARG, "nmodels out of range");
    if (!make_geometry(n, g))
        return ds_fail(ctx, DS_ERR_UNSUPPORTED, "supercell %dx%dx%d: each n must be 1..128 with prime factors 2,3,5,7",
                       n1, n2, n3);
    free_arrays(m);
    free_twiddles(m);
    m->has_occ = m->has_spins = m->has_disp = false;
    m->n[0] = n1;
    m->n[1] = n2;
    m->n[2] = n3;
    m->nmodels = nmodels;
    cudaSetDevice(ctx->device);
    for (int a = 0; a < 3; ++a) {
        CK(cudaMalloc(&m->d_tw32[a], sizeof(c_t<float>) * n[a]));
        CK(cudaMalloc(&m->d_tw64[a], sizeof(c_t<double>) * n[a]));
        make_twiddles<float>(n[a], m->d_tw32[a], 0);
        make_twiddles<double>(n[a], m->d_tw64[a], 0);
    }
    CK(cudaDeviceSynchronize());
    m->has_cells = true;
    return DS_OK;
}

static ds_status upload(ds_model *m, void **dst, const void *src, size_t bytes, int src_dev, void *stream) {
    ds_ctx *ctx = m->ctx;
    if (!src) return ds_fail(ctx, DS_ERR_ARG, "null source array");
    if (!m->has_cells || m->nsite < 1) return ds_fail(ctx, DS_ERR_STATE, "set sites and supercell first");
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    if (!*dst) CK(cudaMalloc(dst, bytes));
    CK(cudaMemcpyAsync(*dst, src, bytes, src_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
    return DS_OK;
}

// after an upload on stream st: mark the model's data ready for requests on any stream, and wait
// for host sources (their memory may be reused by the caller on return)
static ds_status upload_done(ds_model *m, int src_dev, cudaStream_t st) {
    ds_ctx *ctx = m->ctx;
    if (!m->ready) CK(cudaEventCreateWithFlags(&m->ready, cudaEventDisableTiming));
    CK(cudaEventRecord(m->ready, st));
    if (!src_dev) CK(cudaStreamSynchronize(st));
    return DS_OK;
}

static size_t natoms(const ds_model *m) { return (size_t)m->nmodels * m->nsite * m->n[0] * m->n[1] * m->n[2]; }

extern "C" ds_status ds_model_upload_occupancy(ds_model *m, const uint8_t *occ, const double *mean, int src_dev,
                                               void *stream) {
    if (!m) return DS_ERR_ARG;
    ds_status st = upload(m, (void **)&m->d_occ, occ, natoms(m), src_dev, stream);
    if (st != DS_OK) return st;
    ds_ctx *ctx = m->ctx;
    cudaStream_t cs = (cudaStream_t)stream;
    m->has_occ = true;
    m->user_mean = mean != nullptr;
    if (mean) {
        m->mean_occ.assign(mean, mean + m->nsite);
        if (!m->d_user_mean) CK(cudaMalloc(&m->d_user_mean, sizeof(double) * m->nsite));
        CK(cudaMemcpy(m->d_user_mean, mean, sizeof(double) * m->nsite, cudaMemcpyHostToDevice));
    }
    // sample means c_mu over lattice points and supercells (Eq. occ), once per upload
    if (!m->d_mean_occ) CK(cudaMalloc(&m->d_mean_occ, sizeof(double) * m->nsite));
    site_means_occ(m->nmodels, m->nsite, m->n[0] * m->n[1] * m->n[2], m->d_occ, m->d_mean_occ, cs);
    return upload_done(m, src_dev, cs);
}

extern "C" ds_status ds_model_upload_spins(ds_model *m, const float *spins, int src_dev, void *stream) {
    if (!m) return DS_ERR_ARG;
    ds_status st = upload(m, (void **)&m->d_spins, spins, natoms(m) * 3 * sizeof(float), src_dev, stream);
    if (st != DS_OK) return st;
    ds_ctx *ctx = m->ctx;
    cudaStream_t cs = (cudaStream_t)stream;
    m->has_spins = true;
    if (!m->d_mean_spin) CK(cudaMalloc(&m->d_mean_spin, sizeof(double) * 3 * m->nsite));
    site_means_spin(m->nmodels, m->nsite, m->n[0] * m->n[1] * m->n[2], m->d_spins, m->d_mean_spin, cs);
    return upload_done(m, src_dev, cs);
}

extern "C" ds_status ds_model_upload_displacements(ds_model *m, const float *disp, int src_dev, void *stream) {
    if (!m) return DS_ERR_ARG;
    ds_status st = upload(m, (void **)&m->d_disp, disp, natoms(m) * 3 * sizeof(float), src_dev, stream);
    if (st != DS_OK) return st;
    m->has_disp = true;
    return upload_done(m, src_dev, (cudaStream_t)stream);
}

// ------------------------------------------------------------------------------------------
// the forward calculation
// ------------------------------------------------------------------------------------------

ds_status check_request(ds_model *M, const ds_qgrid *q, const ds_opts *o) {
    ds_ctx *ctx = M->ctx;
    if (!q || !o) return ds_fail(ctx, DS_ERR_ARG, "null grid or options");
    if (!M->has_lattice || !M->has_cells || M->nsite < 1) return ds_fail(ctx, DS_ERR_STATE, "model incomplete");
    if (o->precision != DS_FP32 && o->precision != DS_FP64) return ds_fail(ctx, DS_ERR_ARG, "precision");
    if (o->mode != DS_TOTAL && o->mode != DS_DIFFUSE) return ds_fail(ctx, DS_ERR_ARG, "mode");
    if (o->disorder == DS_OCC && !M->has_occ) return ds_fail(ctx, DS_ERR_STATE, "no occupancies uploaded");
    if (o->disorder == DS_SPIN && !M->has_spins) return ds_fail(ctx, DS_ERR_STATE, "no spins uploaded");
    if (o->disorder == DS_DISP && !M->has_disp) return ds_fail(ctx, DS_ERR_STATE, "no displacements uploaded");
    if (o->disorder < 0 || o->disorder > 2) return ds_fail(ctx, DS_ERR_ARG, "disorder");
    if (o->smoothing == DS_SMOOTH_LANCZOS || o->smoothing == DS_SMOOTH_SPHERE) {
        if (o->lanczos_m < 2 || o->lanczos_mprime < 2 || o->lanczos_m * o->lanczos_mprime > 64)
            return ds_fail(ctx, DS_ERR_ARG, "lanczos m, m' must be >= 2 with m m' <= 64");
        if (o->smoothing == DS_SMOOTH_SPHERE && o->lanczos_m * o->lanczos_mprime > 16)
            return ds_fail(ctx, DS_ERR_UNSUPPORTED, "the spherical cutoff handles m m' <= 16");
    } else if (o->smoothing == DS_SMOOTH_SUBBOX) {
        if (o->disorder == DS_DISP)
            return ds_fail(ctx, DS_ERR_UNSUPPORTED, "sub-box averaging is implemented for occupancy and spin disorder");
        for (int a = 0; a < 3; ++a)
            if (o->subbox_n < 1 || 2 * o->subbox_n > M->n[a])
                return ds_fail(ctx, DS_ERR_ARG, "subbox_n must satisfy 1 <= n_sb <= n_alpha/2");
    } else if (o->smoothing != DS_SMOOTH_NONE) {
        return ds_fail(ctx, DS_ERR_ARG, "smoothing");
    }
    if (o->disorder == DS_DISP && o->taylor_order < 0 && !(o->taylor_eps > 0 && o->taylor_eps < 1))
        return ds_fail(ctx, DS_ERR_ARG, "taylor_eps must be in (0, 1) when taylor_order < 0");
    if (o->disorder == DS_DISP && o->taylor_order > 60) return ds_fail(ctx, DS_ERR_UNSUPPORTED, "taylor_order > 60");
    if (o->taylor_zonal != 0 && o->taylor_zonal != 1) return ds_fail(ctx, DS_ERR_ARG, "taylor_zonal must be 0 or 1");
    if (o->dw_coupling != 0 && o->dw_coupling != 1) return ds_fail(ctx, DS_ERR_ARG, "dw_coupling must be 0 or 1");
    if (o->taylor_kernel < DS_TAYLOR_AUTO || o->taylor_kernel > DS_TAYLOR_SUM_FACTORISED)
        return ds_fail(ctx, DS_ERR_ARG, "taylor_kernel");
    if (o->taylor_kernel == DS_TAYLOR_SUM_FACTORISED && o->taylor_zonal)
        return ds_fail(ctx, DS_ERR_UNSUPPORTED, "the sum-factorised Taylor kernel uses one order for the grid");
    if (o->dw_coupling) {
        if (o->disorder != DS_SPIN)
            return ds_fail(ctx, DS_ERR_UNSUPPORTED, "dw_coupling applies to magnetic requests (Eq. mag_sf)");
        if (!M->has_disp) return ds_fail(ctx, DS_ERR_STATE, "dw_coupling needs uploaded displacements");
        if (o->smoothing == DS_SMOOTH_SUBBOX)
            return ds_fail(ctx, DS_ERR_UNSUPPORTED, "dw_coupling is not combined with sub-box averaging");
    }
    if (o->disorder != DS_DISP && M->nsite > 32 && o->disorder == DS_OCC)
        return ds_fail(ctx, DS_ERR_UNSUPPORTED, "occupancy recombination handles up to 32 sites");
    if (o->disorder == DS_SPIN && M->nsite > 16)
        return ds_fail(ctx, DS_ERR_UNSUPPORTED, "magnetic recombination handles up to 16 sites");
    if (o->disorder == DS_DISP && M->nsite > 16)
        return ds_fail(ctx, DS_ERR_UNSUPPORTED, "displacive recombination handles up to 16 sites");
    return DS_OK;
}

// corners of the box of supercell indices [g0, g0 + cnt - 1], as Cartesian Q
void box_corners(const ds_model *M, const int g0[3], const int cnt[3], double corners[24]) {
    int c = 0;
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j)
            for (int l = 0; l < 2; ++l, ++c) {
                const double h = (double)(g0[0] + i * (cnt[0] - 1)) / M->n[0];
                const double k = (double)(g0[1] + j * (cnt[1] - 1)) / M->n[1];
                const double L = (double)(g0[2] + l * (cnt[2] - 1)) / M->n[2];
                for (int a = 0; a < 3; ++a)
                    corners[3 * c + a] = h * M->recip[a] + k * M->recip[3 + a] + L * M->recip[6 + a];
            }
}

// Lanczos resampling with either cutoff (both need the halo of I(G) around the grid)
bool lanczos_like(const ds_opts *o) {
    return o->smoothing == DS_SMOOTH_LANCZOS || o->smoothing == DS_SMOOTH_SPHERE;
}

// |r_c| = (1 - 1/m) |r_max| (2/m' for the variant decaying earlier); |r_max| = the radius of the
// sphere inscribed in the supercell = half the smallest distance n_a 2 pi / |a*_a| between faces
double sphere_cutoff_radius(const ds_model *M, int m, int mprime) {
    const double pi = 3.141592653589793238462643383279502884;
    double rmax = 1e300;
    for (int a = 0; a < 3; ++a) {
        const double bn = sqrt(M->recip[3 * a] * M->recip[3 * a] + M->recip[3 * a + 1] * M->recip[3 * a + 1] +
                               M->recip[3 * a + 2] * M->recip[3 * a + 2]);
        rmax = std::min(rmax, pi * M->n[a] / bn);
    }
    return (1.0 - 1.0 / m) * rmax * 2.0 / mprime;
}

// sin x / x^3 - cos x / x^2 (x = |Q - G| |r_c|), the spherical cutoff without its prefactor
double sphere_profile(double x) {
    if (fabs(x) < 1e-3) return 1.0 / 3.0 - x * x / 30.0;
    return sin(x) / (x * x * x) - cos(x) / (x * x);
}

// normalised (2h+1)^3 stencil of W = W_r(|d|) L(d) over integer offsets d of Bragg positions
void sphere_stencil_weights(const ds_model *M, int m, int mprime, int h, std::vector<double> &w) {
    const double pi = 3.141592653589793238462643383279502884;
    const double meff = 0.5 * m * mprime, rc = sphere_cutoff_radius(M, m, mprime);
    const int nt = 2 * h + 1;
    w.assign((size_t)nt * nt * nt, 0.0);
    auto win = [&](int d) {
        if (!(fabs((double)d) < meff)) return 0.0;
        if (d == 0) return 1.0;
        const double x = pi * d / meff;
        return sin(x) / x;
    };
    double sum = 0.0;
    for (int i = 0; i < nt; ++i)
        for (int j = 0; j < nt; ++j)
            for (int l = 0; l < nt; ++l) {
                const int d[3] = {i - h, j - h, l - h};
                double q[3] = {0, 0, 0};
                for (int a = 0; a < 3; ++a)
                    for (int c = 0; c < 3; ++c) q[c] += (double)d[a] / M->n[a] * M->recip[3 * a + c];
                const double qn = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2]);
                const double v = sphere_profile(qn * rc) * win(d[0]) * win(d[1]) * win(d[2]);
                w[((size_t)i * nt + j) * nt + l] = v;
                sum += v;
            }
    for (double &v : w) v /= sum;
}

// queues the reduction of max |Q.u| over the atoms for the 8 corners of the computing grid (the
// requested grid plus the Lanczos halo) and max |u|, and their copy into host_out[9] (pinned or
// pageable host memory; valid once stream st reaches this point)
ds_status queue_corner_xmax(ds_model *M, const ds_qgrid *q, const ds_opts *o, cudaStream_t st, Scratch &ws,
                            double *host_out) {
    ds_ctx *ctx = M->ctx;
    int g0[3], cnt[3];
    ds_status rc = grid_indices(ctx, M, q, g0, cnt);
    if (rc != DS_OK) return rc;
    const int halo = lanczos_like(o) ? lanczos_halo(o->lanczos_m, o->lanczos_mprime) : 0;
    int eg0[3], ecnt[3];
    for (int a = 0; a < 3; ++a) {
        eg0[a] = g0[a] - halo;
        ecnt[a] = cnt[a] + 2 * halo;
    }
    Corners corners;
    box_corners(M, eg0, ecnt, corners.v);
    if (M->ready) CK(wait_unless_done(st, M->ready));
    double *d_x = (double *)ws.get(sizeof(double) * 9);
    if (ws.failed) return ds_fail(ctx, DS_ERR_OOM, "device allocation failed");
    const size_t natom = (size_t)M->nmodels * M->nsite * M->n[0] * M->n[1] * M->n[2];
    corner_xmax((int)natom, M->d_disp, corners, d_x, st);
    CK(cudaMemcpyAsync(host_out, d_x, sizeof(double) * 9, cudaMemcpyDeviceToHost, st));
    return DS_OK;
}

// the Taylor order of Section III C from the corner maxima hx[9] (see queue_corner_xmax)
ds_status taylor_order_from_corners(ds_ctx *ctx, const ds_opts *o, const double hx[9], int *P, double *xmax,
                                    double *umax) {
    double x = 0.0;
    for (int c = 0; c < 8; ++c) x = std::max(x, hx[c]);
    *xmax = x;
    if (umax) *umax = hx[8];
    *P = taylor_order_for(x, o->taylor_eps);
    if (*P < 0 || *P > 60) return ds_fail(ctx, DS_ERR_UNSUPPORTED, "Taylor order above 60 (x_max = %g)", x);
    return DS_OK;
}

// smallest order whose remainder bound x_max^(P+1)/(P+1)! <= eps over the computing grid
// (the requested grid plus the Lanczos halo); reads x_max back from the device (synchronises st)
ds_status resolve_taylor_order(ds_model *M, const ds_qgrid *q, const ds_opts *o, cudaStream_t st, Scratch &ws, int *P,
                               double *xmax, double *umax) {
    ds_ctx *ctx = M->ctx;
    double hx[9];
    ds_status rc = queue_corner_xmax(M, q, o, st, ws, hx);
    if (rc != DS_OK) return rc;
    CK(cudaStreamSynchronize(st));
    return taylor_order_from_corners(ctx, o, hx, P, xmax, umax);
}

// device bytes a request takes from the pool (the caller's output excluded); P = Taylor order
size_t request_footprint(const ds_model *M, const ds_qgrid *q, const ds_opts *o, int P) {
    Geometry g;
    make_geometry(M->n, g);
    const size_t es = o->precision == DS_FP64 ? 8 : 4, ce = 2 * es;
    const size_t nsite = M->nsite, nmod = M->nmodels;
    size_t cnt[3];
    for (int a = 0; a < 3; ++a) cnt[a] = (size_t)q->count[a];
    size_t bytes = 64 * 1024;  // tables
    if (o->smoothing == DS_SMOOTH_SUBBOX) {
        const size_t nf = nsite * (o->disorder == DS_SPIN ? 3 : 1), npair = nf * (nf + 1) / 2;
        bytes += nmod * nf * g.ncell * es + npair * g.ncell * es + 2 * npair * g.ncell_h * ce;
        return bytes;
    }
    size_t nf = nmod * nsite;
    if (o->disorder == DS_SPIN) nf *= 3;
    if (o->disorder == DS_DISP) {
        const size_t T = (size_t)(P + 1) * (P + 2) * (P + 3) / 6;
        nf *= T;
        bytes += nmod * nsite * g.ncell * 3 * (P + 1) * es;
    }
    const size_t fb = std::max<size_t>(1, std::min<size_t>(nf, (512ull << 20) / (ce * g.ncell_h)));
    bytes += (nf + fb) * g.ncell_h * ce;
    const int hl = lanczos_like(o) ? lanczos_halo(o->lanczos_m, o->lanczos_mprime) : 0;
    if (lanczos_like(o)) bytes += 3 * (cnt[0] + 2 * hl) * (cnt[1] + 2 * hl) * (cnt[2] + 2 * hl) * es;
    if (o->dw_coupling) bytes += nsite * (cnt[0] + 2 * hl) * (cnt[1] + 2 * hl) * (cnt[2] + 2 * hl) * es;
    return bytes;
}

// residue classes of zones along each axis (the period of exp(2 pi i H_a r_mu,a), or every zone its
// own class); dres stays 0 unless the classes are at most half as many as the zones
bool residue_classes(const ds_model *M, const GridMap &gm, int dres[3]) {
    int d[3];
    for (int a = 0; a < 3; ++a) d[a] = (M->period[a] > 0 && M->period[a] < gm.nH[a]) ? M->period[a] : gm.nH[a];
    if (2LL * d[0] * d[1] * d[2] > (long long)gm.nH[0] * gm.nH[1] * gm.nH[2]) return false;
    for (int a = 0; a < 3; ++a) dres[a] = d[a];
    return true;
}

// site phase tables exp(2 pi i k_a r_a / n_a) and exp(2 pi i H_a r_a) of a grid, cached per model
// (at most 256 grids; beyond that they are rebuilt in request scratch); a stream that did not
// build them waits for the building stream's kernel
template <typename T>
ds_status site_tables(ds_model *M, const Geometry &g, const GridMap &gm, int nmax, int nHmax, cudaStream_t st,
                      Scratch &ws, const c_t<T> **phk, const c_t<T> **phH) {
    using C = c_t<T>;
    ds_ctx *ctx = M->ctx;
    const std::vector<int> key = {(int)sizeof(T), gm.Hmin[0], gm.Hmin[1], gm.Hmin[2], gm.nH[0], gm.nH[1], gm.nH[2]};
    const size_t bk = sizeof(C) * M->nsite * 3 * nmax, bh = sizeof(C) * M->nsite * 3 * nHmax;
    std::lock_guard<std::mutex> lk(M->cache_mu);
    auto it = M->site_tables.find(key);
    if (it != M->site_tables.end()) {
        CK(wait_unless_done(st, it->second.done));
        *phk = (const C *)it->second.phk;
        *phH = (const C *)it->second.phH;
        return DS_OK;
    }
    C *k = nullptr, *h = nullptr;
    if (M->site_tables.size() >= 256) {
        k = (C *)ws.get(bk);
        h = (C *)ws.get(bh);
        if (ws.failed) return ds_fail(ctx, DS_ERR_OOM, "device allocation failed (tables)");
        make_site_tables<T>(g, gm, M->nsite, M->d_sites, k, h, nmax, nHmax, st);
    } else {
        ds_model::SiteTables e;
        CK(cudaMalloc(&e.phk, bk));
        CK(cudaMalloc(&e.phH, bh));
        CK(cudaEventCreateWithFlags(&e.done, cudaEventDisableTiming));
        make_site_tables<T>(g, gm, M->nsite, M->d_sites, (C *)e.phk, (C *)e.phH, nmax, nHmax, st);
        CK(cudaEventRecord(e.done, st));
        M->site_tables[key] = e;
        k = (C *)e.phk;
        h = (C *)e.phH;
    }
    *phk = k;
    *phH = h;
    return DS_OK;
}

template <typename T>
ds_status plan_and_run(ds_model *M, const ds_qgrid *q, const ds_opts *o, T *d_out, cudaStream_t st, Scratch &ws,
                       ds_result_info *info, ForwardKeep<T> *keep, const TaylorHint *hint) {
    using C = c_t<T>;
    ds_ctx *ctx = M->ctx;
    int g0[3], cnt[3];
    ds_status rc = grid_indices(ctx, M, q, g0, cnt);
    if (rc != DS_OK) return rc;
    if (M->ready) CK(wait_unless_done(st, M->ready));  // uploads made on another stream
    Geometry g;
    make_geometry(M->n, g);
    const int nsite = M->nsite, nmod = M->nmodels;
    const size_t natom = (size_t)nmod * nsite * g.ncell;

    // computing grid: extended by the Lanczos halo on every side
    int halo = 0;
    if (lanczos_like(o)) halo = lanczos_halo(o->lanczos_m, o->lanczos_mprime);
    int eg0[3], ecnt[3];
    for (int a = 0; a < 3; ++a) {
        eg0[a] = g0[a] - halo;
        ecnt[a] = cnt[a] + 2 * halo;
    }
    const GridMap gm = grid_map(g, eg0, ecnt);

    RecombParams<T> p;
    memset(&p, 0, sizeof(p));
    p.g = g;
    p.gm = gm;
    p.nsite = nsite;
    p.nmodels = nmod;
    p.diffuse = o->mode == DS_DIFFUSE;
    if (!M->ff_ok) return ds_fail(ctx, DS_ERR_UNSUPPORTED, "more than %d distinct form factors", MAX_FF_CLASSES);
    if constexpr (sizeof(T) == 4) p.ff = M->ff32;
    else p.ff = M->ff64;
    p.grp = M->groups;
    if (o->disorder != DS_DISP) residue_classes(M, gm, p.dres);
    set_reciprocal(p, M->recip, g.n);
    const double N = (double)nsite * g.ncell;
    p.norm = (T)(1.0 / (nmod * N));
    if (o->disorder == DS_SPIN) p.norm = (T)(0.07265 / (nmod * N));  // C of Eq. mag_intensity (barn)

    // small tables: site phases of this grid (twiddles, site order and b are per model)
    p.nmax = std::max(g.n[0], std::max(g.n[1], g.n[2]));
    p.nHmax = std::max(gm.nH[0], std::max(gm.nH[1], gm.nH[2]));
    const C *W[3];
    for (int a = 0; a < 3; ++a) {
        if constexpr (sizeof(T) == 4) W[a] = M->d_tw32[a];
        else W[a] = M->d_tw64[a];
    }
    rc = site_tables<T>(M, g, gm, p.nmax, p.nHmax, st, ws, &p.phk, &p.phH);
    if (rc != DS_OK) return rc;
    p.site_of = M->d_site_of;
    p.sites = M->d_sites;
    if constexpr (sizeof(T) == 4) p.scat = M->d_scat32;
    else p.scat = M->d_scat64;
    p.out = d_out;

    FieldSource src;
    memset(&src, 0, sizeof(src));
    src.nsite = nsite;
    src.diffuse = o->mode == DS_DIFFUSE;
    int nf_model = 0;
    int P = 0, Tn = 1;
    double xmax = -1.0;
    if (o->disorder == DS_OCC) {
        src.kind = SRC_OCC;
        src.occ = M->d_occ;
        nf_model = nsite;
        src.mean = M->user_mean ? M->d_user_mean : M->d_mean_occ;
        p.ncomp = 1;
    } else if (o->disorder == DS_SPIN) {
        src.kind = SRC_SPIN;
        src.vec3 = M->d_spins;
        nf_model = 3 * nsite;
        src.mean = M->d_mean_spin;
        p.ncomp = 3;
    } else {
        // coefficient scales: the largest |g_a| = |G_a| / n_a over the computing grid, so that the
        // scaled coefficients x1^a x2^b x3^c stay within [-1, 1]
        double gscale[3];
        for (int a = 0; a < 3; ++a) {
            gscale[a] = std::max(fabs((double)eg0[a]), fabs((double)eg0[a] + ecnt[a] - 1)) / g.n[a];
            if (!(gscale[a] > 0)) gscale[a] = 1.0;
        }
        P = o->taylor_order;
        double umax = 0.0;
        const bool auto_order = P < 0;
        if (auto_order && hint) {
            P = hint->P;
            xmax = hint->xmax;
            umax = hint->umax;
        } else if (auto_order) {
            rc = resolve_taylor_order(M, q, o, st, ws, &P, &xmax, &umax);
            if (rc != DS_OK) return rc;
        }
        int4 *d_terms = nullptr;
        int *d_ops = nullptr;
        rc = taylor_tables(M, P, &d_terms, &d_ops, &Tn);
        if (rc != DS_OK) return rc;
        T *pw = (T *)ws.get(sizeof(T) * natom * 3 * (P + 1));
        if (ws.failed) return ds_fail(ctx, DS_ERR_OOM, "device allocation failed (power tables)");
        make_powers<T>(g, nmod, nsite, P, M->recip, gscale, M->d_disp, pw, st);
        src.kind = SRC_DISP;
        src.pw = pw;
        src.terms = d_terms;
        src.T = Tn;
        src.P = P;
        src.occ = M->has_occ ? M->d_occ : nullptr;
        nf_model = nsite * Tn;
        p.ncomp = 1;
        p.nT = Tn;
        p.ops = d_ops;
        p.terms = d_terms;
        for (int a = 0; a < 3; ++a) p.gscale[a] = gscale[a];
        if (auto_order && o->taylor_zonal && P > 0) {
            // Taylor order per zone: every voxel G of a zone has max_j |Q.u_j| <= min(|Q|max u_max,
            // x_max) (Cauchy-Schwarz), so the remainder bound of Section III C holds there with the
            // order of that smaller argument; |Q| is convex, its maximum over the zone's voxel box
            // is at a corner
            const int nz = gm.nH[0] * gm.nH[1] * gm.nH[2];
            std::vector<int> pz(nz);
            for (int h1 = 0; h1 < gm.nH[0]; ++h1)
                for (int h2 = 0; h2 < gm.nH[1]; ++h2)
                    for (int h3 = 0; h3 < gm.nH[2]; ++h3) {
                        const int hh[3] = {h1, h2, h3};
                        int lo[3], hi[3];
                        for (int a = 0; a < 3; ++a) {
                            const int H = gm.Hmin[a] + hh[a];
                            lo[a] = std::max(g.n[a] * H, gm.g0[a]);
                            hi[a] = std::min(g.n[a] * (H + 1) - 1, gm.g0[a] + gm.cnt[a] - 1);
                        }
                        double qmax = 0.0;
                        for (int c = 0; c < 8; ++c) {
                            const double Gc[3] = {(double)((c & 4) ? hi[0] : lo[0]) / g.n[0],
                                                  (double)((c & 2) ? hi[1] : lo[1]) / g.n[1],
                                                  (double)((c & 1) ? hi[2] : lo[2]) / g.n[2]};
                            double Qc[3];
                            for (int a = 0; a < 3; ++a)
                                Qc[a] = Gc[0] * M->recip[a] + Gc[1] * M->recip[3 + a] + Gc[2] * M->recip[6 + a];
                            qmax = std::max(qmax, sqrt(Qc[0] * Qc[0] + Qc[1] * Qc[1] + Qc[2] * Qc[2]));
                        }
                        const double xz = std::min(qmax * umax, xmax);
                        pz[((size_t)h1 * gm.nH[1] + h2) * gm.nH[2] + h3] = std::min(P, taylor_order_for(xz, o->taylor_eps));
                    }
            int *d_pz = (int *)ws.get(sizeof(int) * nz);
            int *tab = nullptr;
            if (ws.failed) return ds_fail(ctx, DS_ERR_OOM, "device allocation failed (zone orders)");
            rc = sub_simplex_tables(M, P, &tab);
            if (rc != DS_OK) return rc;
            CK(cudaMemcpyAsync(d_pz, pz.data(), sizeof(int) * nz, cudaMemcpyHostToDevice, st));
            const size_t nsub = (size_t)(P + 1) * (P + 2) * (P + 3) * (P + 4) / 24;
            p.pzone = d_pz;
            p.sub_map = tab;
            p.sub_ops = tab + nsub;
            p.sub_off = tab + 2 * nsub;
        }
        if (keep) {
            keep->terms = d_terms;
            keep->pw = pw;
        }
    }
    src.nf_per_model = nf_model;
    const int nf = nf_model * nmod;

    // displacive with one order for the grid: the sum-factorised recombination (taylor_sf.cu), with
    // zone phases over the grid's zones and those of its negation (Friedel mates)
    bool use_sf = false;
    if (o->disorder == DS_DISP && !p.pzone && o->taylor_kernel != DS_TAYLOR_PER_VOXEL) {
        std::vector<int4> items;
        const bool force = o->taylor_kernel == DS_TAYLOR_SUM_FACTORISED;
        const bool ok = taylor_sf_plan(g, gm, P, nsite, sizeof(C), force, p.sf, items);
        if (force && !ok)
            return ds_fail(ctx, DS_ERR_UNSUPPORTED, "sum-factorised Taylor kernel: zone boxes wider than 17 per axis");
        if (ok) {
            GridMap gmx = gm;
            int nHx = 1;
            for (int a = 0; a < 3; ++a) {
                const int Hmax = gm.Hmin[a] + gm.nH[a] - 1;
                gmx.Hmin[a] = std::min(gm.Hmin[a], -Hmax - 1);
                gmx.nH[a] = std::max(Hmax, -gm.Hmin[a]) - gmx.Hmin[a] + 1;
                nHx = std::max(nHx, gmx.nH[a]);
            }
            const C *phk2 = nullptr;
            rc = site_tables<T>(M, g, gmx, p.nmax, nHx, st, ws, &phk2, &p.phHx);
            if (rc != DS_OK) return rc;
            for (int a = 0; a < 3; ++a) p.Hminx[a] = gmx.Hmin[a];
            p.nHx = nHx;
            int4 *d_items = (int4 *)ws.get(sizeof(int4) * items.size());
            if (ws.failed) return ds_fail(ctx, DS_ERR_OOM, "device allocation failed (Taylor plan)");
            CK(cudaMemcpyAsync(d_items, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice, st));
            p.sf.items = d_items;
            use_sf = true;
        }
    }

    // per-site transforms (Section III)
    C *spec = (C *)ws.get(sizeof(C) * (size_t)nf * g.ncell_h);
    const size_t work_cap = 512ull << 20;
    int fb = (int)std::max<size_t>(1, std::min<size_t>(nf, work_cap / (sizeof(C) * (size_t)g.ncell_h)));
    C *work = (C *)ws.get(sizeof(C) * (size_t)fb * g.ncell_h);
    if (ws.failed) return ds_fail(ctx, DS_ERR_OOM, "device allocation failed (spectra: %zu bytes)",
                                  sizeof(C) * (size_t)nf * g.ncell_h);
    if (ws.total > ctx->budget)
        return ds_fail(ctx, DS_ERR_ADMISSION, "request needs %zu bytes of scratch, budget %zu", ws.total, ctx->budget);
    {
        ProfScope ps(ctx, "fft", st);
        for (int f0 = 0; f0 < nf; f0 += fb)
            fft_real_fields<T>(g, src, f0, std::min(fb, nf - f0), work, spec, W[0], W[1], W[2], st);
    }
    p.spec = spec;

    // recombination over the requested voxels (+ Bragg term)
    if (keep && keep->Fout) {
        p.Fout = keep->Fout;
        p.force_plain = 1;
    }
    if (o->disorder == DS_SPIN && o->dw_coupling) {
        // T_mu(G) per voxel and site breaks the sharing of site sums across zones: plain kernel
        T *dw = (T *)ws.get(sizeof(T) * (size_t)nsite * ecnt[0] * ecnt[1] * ecnt[2]);
        if (ws.failed) return ds_fail(ctx, DS_ERR_OOM, "device allocation failed (Debye-Waller factors)");
        ProfScope ps(ctx, "debye_waller", st);
        debye_waller_grid<T>(M, eg0, ecnt, dw, st);
        p.dw = dw;
        p.force_plain = 1;
    }
    if (o->disorder == DS_DISP) {
        if (p.diffuse) {
            C *avg0 = (C *)ws.get(sizeof(C) * nsite * Tn);
            C *bragg = (C *)ws.get(sizeof(C) * (size_t)gm.nH[0] * gm.nH[1] * gm.nH[2]);
            if (ws.failed) return ds_fail(ctx, DS_ERR_OOM, "device allocation failed");
            ProfScope ps(ctx, "bragg_disp", st);
            displacive_bragg<T>(p, src.terms, avg0, bragg, st);
            p.bragg = bragg;
        }
        ProfScope ps(ctx, "recombine_disp", st);
        for (int m = 0; m < nmod; ++m) {
            p.model = m;
            p.accumulate = m > 0;
            if (use_sf) recombine_disp_sf<T>(p, st);
            else recombine_disp<T>(p, st);
        }
    } else {
        ProfScope ps(ctx, p.ncomp == 1 ? "recombine_occ" : "recombine_spin", st);
        for (int m = 0; m < nmod; ++m) {
            p.model = m;
            p.accumulate = m > 0;
            recombine_cm<T>(p, st);
        }
    }
    CK(cudaGetLastError());
    if (keep) {
        keep->p = p;
        keep->g = g;
        keep->src = src;
        keep->W[0] = W[0];
        keep->W[1] = W[1];
        keep->W[2] = W[2];
    }
    if (info) {
        info->taylor_order = P;
        info->n_monomials = o->disorder == DS_DISP ? Tn : 0;
        info->x_max = xmax;
        info->trunc_bound = (o->disorder == DS_DISP && xmax >= 0)
                                ? exp((P + 1) * log(std::max(xmax, 1e-300)) - lgamma((double)P + 2.0))
                                : 0.0;
    }
    return DS_OK;
}

// the request's kernels on stream st into the device volume d_out (no synchronisation)
template <typename T>
ds_status enqueue_request(ds_model *M, const ds_qgrid *q, const ds_opts *o, T *d_out, cudaStream_t st, Scratch &ws,
                          ds_result_info *info, const TaylorHint *hint) {
    ds_ctx *ctx = M->ctx;
    int g0[3], cnt[3];
    ds_status rc = grid_indices(ctx, M, q, g0, cnt);
    if (rc != DS_OK) return rc;
    if (o->smoothing == DS_SMOOTH_SUBBOX) {
        rc = subbox_run<T>(M, q, o, d_out, st, ws, info);
    } else if (o->smoothing == DS_SMOOTH_LANCZOS) {
        const int h = lanczos_halo(o->lanczos_m, o->lanczos_mprime);
        const size_t next = (size_t)(cnt[0] + 2 * h) * (cnt[1] + 2 * h) * (cnt[2] + 2 * h);
        T *ext = (T *)ws.get(sizeof(T) * next);
        T *t1 = (T *)ws.get(sizeof(T) * next);
        T *t2 = (T *)ws.get(sizeof(T) * next);
        if (ws.failed) return ds_fail(ctx, DS_ERR_OOM, "device allocation failed (Lanczos buffers)");
        rc = plan_and_run<T>(M, q, o, ext, st, ws, info, nullptr, hint);
        if (rc == DS_OK) {
            ProfScope ps(ctx, "lanczos", st);
            lanczos_resample<T>(ext, t1, t2, d_out, cnt, o->lanczos_m, o->lanczos_mprime, st);
        }
    } else if (o->smoothing == DS_SMOOTH_SPHERE) {
        const int h = lanczos_halo(o->lanczos_m, o->lanczos_mprime);
        const size_t next = (size_t)(cnt[0] + 2 * h) * (cnt[1] + 2 * h) * (cnt[2] + 2 * h);
        const int nt = 2 * h + 1;
        T *ext = (T *)ws.get(sizeof(T) * next);
        T *dw = (T *)ws.get(sizeof(T) * nt * nt * nt);
        if (ws.failed) return ds_fail(ctx, DS_ERR_OOM, "device allocation failed (resampling buffers)");
        std::vector<double> w;
        sphere_stencil_weights(M, o->lanczos_m, o->lanczos_mprime, h, w);
        std::vector<T> wt(w.begin(), w.end());
        CK(cudaMemcpyAsync(dw, wt.data(), sizeof(T) * wt.size(), cudaMemcpyHostToDevice, st));
        rc = plan_and_run<T>(M, q, o, ext, st, ws, info, nullptr, hint);
        if (rc == DS_OK) {
            ProfScope ps(ctx, "lanczos_sphere", st);
            sphere_resample<T>(ext, dw, d_out, cnt, h, st);
        }
        // the host weights must outlive their asynchronous copy
        CK(cudaStreamSynchronize(st));
    } else {
        rc = plan_and_run<T>(M, q, o, d_out, st, ws, info, nullptr, hint);
    }
    if (rc == DS_OK && info) {
        info->nvox = (int64_t)cnt[0] * cnt[1] * cnt[2];
        info->workspace_bytes = (int64_t)ws.total;
    }
    return rc;
}

template <typename T>
static ds_status run_intensity(ds_model *M, const ds_qgrid *q, const ds_opts *o, void *out, int out_dev,
                               cudaStream_t st, ds_result_info *info) {
    ds_ctx *ctx = M->ctx;
    int g0[3], cnt[3];
    ds_status rc = grid_indices(ctx, M, q, g0, cnt);
    if (rc != DS_OK) return rc;
    const size_t nvox = (size_t)cnt[0] * cnt[1] * cnt[2];
    Scratch ws(st);
    T *d_out = out_dev ? (T *)out : (T *)ws.get(sizeof(T) * nvox);
    if (!d_out) return ds_fail(ctx, DS_ERR_OOM, "device allocation failed (output)");
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (!out_dev) {
        CK(cudaEventCreate(&e0));
        CK(cudaEventCreate(&e1));
        cudaEventRecord(e0, st);
    }
    if (info) info->gpu_ms = 0.0;
    rc = enqueue_request<T>(M, q, o, d_out, st, ws, info);
    if (rc == DS_OK && !out_dev) {
        cudaEventRecord(e1, st);
        if (cudaMemcpyAsync(out, d_out, sizeof(T) * nvox, cudaMemcpyDeviceToHost, st) != cudaSuccess)
            rc = ds_fail(ctx, DS_ERR_CUDA, "copy of the volume to the host failed");
    }
    ws.release();
    if (!out_dev || rc != DS_OK) {
        if (cudaStreamSynchronize(st) != cudaSuccess && rc == DS_OK)
            rc = ds_fail(ctx, DS_ERR_CUDA, "stream synchronisation failed: %s", cudaGetErrorString(cudaGetLastError()));
    }
    if (e0) {
        float ms = 0.f;
        if (rc == DS_OK && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && info) info->gpu_ms = ms;
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
    }
    if (rc != DS_OK) return rc;
    CK(cudaGetLastError());
    return DS_OK;
}

extern "C" ds_status ds_request_intensity(ds_model *M, const ds_qgrid *q, const ds_opts *o, void *out,
                                          int out_is_device, void *stream, ds_result_info *info) {
    if (!M) return DS_ERR_ARG;
    ds_ctx *ctx = M->ctx;
    if (!out) return ds_fail(ctx, DS_ERR_ARG, "null output");
    ds_status rc = check_request(M, q, o);
    if (rc != DS_OK) return rc;
    CK(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    if (o->precision == DS_FP64) return run_intensity<double>(M, q, o, out, out_is_device, st, info);
    return run_intensity<float>(M, q, o, out, out_is_device, st, info);
}

template ds_status plan_and_run<float>(ds_model *, const ds_qgrid *, const ds_opts *, float *, cudaStream_t,
                                       Scratch &, ds_result_info *, ForwardKeep<float> *, const TaylorHint *);
template ds_status plan_and_run<double>(ds_model *, const ds_qgrid *, const ds_opts *, double *, cudaStream_t,
                                        Scratch &, ds_result_info *, ForwardKeep<double> *, const TaylorHint *);

// ------------------------------------------------------------------------------------------
// tracing
// ------------------------------------------------------------------------------------------

static std::atomic<long long> g_launches{0};
void ds::count_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

static cudaEvent_t pool_event(ds_ctx *ctx) {
    std::lock_guard<std::mutex> g(ctx->prof_mu);
    if (ctx->event_pool.empty()) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        return e;
    }
    cudaEvent_t e = ctx->event_pool.back();
    ctx->event_pool.pop_back();
    return e;
}

ProfScope::ProfScope(ds_ctx *c, const char *name, cudaStream_t st) : ctx(c), s(st), on(c && c->prof_on) {
    if (!on) return;
    rec.name = name;
    rec.e0 = pool_event(ctx);
    rec.e1 = pool_event(ctx);
    cudaEventRecord(rec.e0, s);
}
ProfScope::~ProfScope() {
    if (!on) return;
    cudaEventRecord(rec.e1, s);
    std::lock_guard<std::mutex> g(ctx->prof_mu);
    ctx->prof.push_back(rec);
}

extern "C" ds_status ds_profile_enable(ds_ctx *ctx, int enable) {
    if (!ctx) return DS_ERR_ARG;
    ctx->prof_on = enable != 0;
    return DS_OK;
}

extern "C" ds_status ds_profile_report(ds_ctx *ctx, char *json, size_t cap) {
    if (!ctx || !json) return DS_ERR_ARG;
    std::vector<ProfRecord> recs;
    {
        std::lock_guard<std::mutex> g(ctx->prof_mu);
        recs.swap(ctx->prof);
    }
    std::vector<std::string> names;
    std::vector<double> ms;
    std::vector<long> cnt;
    cudaSetDevice(ctx->device);
    ds_status rc = DS_OK;
    for (auto &r : recs) {
        float t = 0.f;
        if (cudaEventSynchronize(r.e1) != cudaSuccess || cudaEventElapsedTime(&t, r.e0, r.e1) != cudaSuccess)
            rc = DS_ERR_CUDA;
        size_t i = 0;
        while (i < names.size() && names[i] != r.name) ++i;
        if (i == names.size()) {
            names.push_back(r.name);
            ms.push_back(0.0);
            cnt.push_back(0);
        }
        ms[i] += t;
        cnt[i] += 1;
    }
    {
        std::lock_guard<std::mutex> g(ctx->prof_mu);
        for (auto &r : recs) {
            ctx->event_pool.push_back(r.e0);
            ctx->event_pool.push_back(r.e1);
        }
    }
    std::string out = "{\"stages\": {";
    for (size_t i = 0; i < names.size(); ++i) {
        char buf[256];
        snprintf(buf, sizeof(buf), "%s\"%s\": {\"count\": %ld, \"ms\": %.6f}", i ? ", " : "", names[i].c_str(), cnt[i],
                 ms[i]);
        out += buf;
    }
    char tail[64];
    snprintf(tail, sizeof(tail), "}, \"launches\": %lld}", g_launches.exchange(0));
    out += tail;
    if (out.size() + 1 > cap) return ds_fail(ctx, DS_ERR_ARG, "profile buffer too small (%zu bytes needed)", out.size() + 1);
    memcpy(json, out.c_str(), out.size() + 1);
    if (rc != DS_OK) return ds_fail(ctx, rc, "event timing failed");
    return DS_OK;
}

template ds_status enqueue_request<float>(ds_model *, const ds_qgrid *, const ds_opts *, float *, cudaStream_t,
                                          Scratch &, ds_result_info *, const TaylorHint *);
template ds_status enqueue_request<double>(ds_model *, const ds_qgrid *, const ds_opts *, double *, cudaStream_t,
                                           Scratch &, ds_result_info *, const TaylorHint *);
