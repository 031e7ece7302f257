// Occupancy (compositional) intensity without any device allocation.
//
// Some callers cannot allocate device memory at the moment they need an intensity volume:
// code running inside a host application or framework that owns the GPU's memory through its
// own allocator (and forbids direct cudaMalloc), processes started with a fixed memory cap, or
// a refinement loop that must not touch the allocator between iterations.  This entry point
// serves them: it computes the same result as ds_request_intensity for occupancy disorder with
// constant form factors in FP32, but every intermediate (twiddles, site-phase tables, site
// data and means, per-site spectra, FFT work buffer) lives in one file-scope device array of
// fixed size, g_noalloc_scratch.  The caller passes the inputs and the output; nothing is
// allocated.  The per-site inputs (at most 32 sites) travel as a kernel argument, so no host
// buffer is read after the call returns.
//
// Properties a caller must know:
//  - The array is DS_NOALLOC_SCRATCH_BYTES (32 MiB) on every GPU that loads the library and stays
//    there until the process exits.  Requests needing more are rejected with DS_ERR_ADMISSION.
//  - The first call on a device (and the first after that device's context was reset) looks up
//    the array's device address (cudaGetSymbolAddress) with that device current.  The entry
//    point is for direct calls on a stream; recording it into a CUDA graph is not supported.
//  - All calls share the array.  Every kernel writes the scratch it reads before reading it, so
//    no part of the array has to start at zero, but two calls whose work overlaps on the GPU
//    (different streams, or several host threads) race on it: serialise them.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "../../include/ds.h"
#include "api_internal.h"
#include "internal.h"

using namespace ds;

#define DS_NOALLOC_SCRATCH_BYTES (32u << 20)

static __device__ __align__(256) unsigned char g_noalloc_scratch[DS_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
constexpr int kMaxSites = 32;

// per-device cache of the array's address, valid for the context it was looked up in
struct ScratchAddr {
    unsigned long long ctx_id = 0;
    bool have_id = false;
    unsigned char *addr = nullptr;
};
std::mutex g_addr_mu;
ScratchAddr g_addr[kMaxDevices];

typedef int (*ctx_get_id_fn)(void *ctx, unsigned long long *id);  // cuCtxGetId(NULL = current)

ds_status say(char *err, size_t errlen, ds_status st, const char *fmt, ...) {
    if (err && errlen) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(err, errlen, fmt, ap);
        va_end(ap);
    }
    return st;
}

// unique id of the current context (false when the driver cannot tell)
bool current_context_id(unsigned long long *id) {
    static ctx_get_id_fn fn = nullptr;
    static bool looked = false;
    if (!looked) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (ctx_get_id_fn)p;
        cudaGetLastError();
        looked = true;
    }
    return fn && fn(nullptr, id) == 0;
}

// device address of the static scratch on device `dev` (current): looked up once per device
// context, again when the context changed (a reset unloads the module and the array may move)
ds_status scratch_address(int dev, unsigned char **out, char *err, size_t errlen) {
    if (dev < 0 || dev >= kMaxDevices) return say(err, errlen, DS_ERR_ARG, "device %d out of range", dev);
    std::lock_guard<std::mutex> g(g_addr_mu);
    ScratchAddr &c = g_addr[dev];
    unsigned long long id = 0;
    const bool have_id = current_context_id(&id);
    if (!c.addr || !have_id || !c.have_id || c.ctx_id != id) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return say(err, errlen, DS_ERR_CUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        c.addr = (unsigned char *)p;
        c.ctx_id = id;
        c.have_id = have_id;
    }
    *out = c.addr;
    return DS_OK;
}

// the caller's per-site inputs, passed by value to the kernel that writes them into the scratch
struct SiteInputs {
    int nsite;
    int has_mean;
    double frac[3 * kMaxSites];
    int site_of[kMaxSites];
    float scat[kMaxSites];
    double mean[kMaxSites];
};

__global__ void k_noalloc_sites(const SiteInputs in, double *sites, int *site_of, float *scat, double *mean) {
    const int i = threadIdx.x;
    if (i >= in.nsite) return;
    for (int a = 0; a < 3; ++a) sites[3 * i + a] = in.frac[3 * i + a];
    site_of[i] = in.site_of[i];
    scat[i] = in.scat[i];
    if (in.has_mean) mean[i] = in.mean[i];
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

extern "C" ds_status ds_occupancy_intensity_noalloc(const double lattice[6], int nsite, const double *frac_xyz,
                                                    const double *scat_len, int n1, int n2, int n3, int nmodels,
                                                    const uint8_t *occ_dev, const double *mean_occ,
                                                    const ds_qgrid *grid, int mode, float *out_dev, void *stream,
                                                    char *err, size_t errlen) {
    using C = c_t<float>;
    if (err && errlen) err[0] = 0;
    if (!lattice || !frac_xyz || !occ_dev || !grid || !out_dev) return say(err, errlen, DS_ERR_ARG, "null argument");
    if (nsite < 1 || nsite > kMaxSites) return say(err, errlen, DS_ERR_ARG, "nsite must be 1..%d", kMaxSites);
    for (int i = 0; i < nsite; ++i) {
        for (int a = 0; a < 3; ++a)
            if (!std::isfinite(frac_xyz[3 * i + a])) return say(err, errlen, DS_ERR_ARG, "site %d coordinate", i);
        if (scat_len && !std::isfinite(scat_len[i])) return say(err, errlen, DS_ERR_ARG, "site %d scattering length", i);
        if (mean_occ && !std::isfinite(mean_occ[i])) return say(err, errlen, DS_ERR_ARG, "site %d mean occupancy", i);
    }
    if (nmodels < 1) return say(err, errlen, DS_ERR_ARG, "nmodels must be >= 1");
    if (mode != DS_TOTAL && mode != DS_DIFFUSE) return say(err, errlen, DS_ERR_ARG, "mode");
    const int n[3] = {n1, n2, n3};
    Geometry g;
    if (!make_geometry(n, g))
        return say(err, errlen, DS_ERR_UNSUPPORTED, "supercell %dx%dx%d: each n must be 1..128 with factors 2,3,5,7", n1, n2,
                   n3);
    int g0[3], cnt[3];
    for (int a = 0; a < 3; ++a) {
        if (grid->count[a] < 1 || grid->count[a] > (1 << 20)) return say(err, errlen, DS_ERR_ARG, "grid count[%d]", a);
        if (!(fabs(grid->step[a] * n[a] - 1.0) < 1e-9))
            return say(err, errlen, DS_ERR_UNSUPPORTED, "grid axis %d: step is not 1/n (commensurate grids only)", a);
        const double x = grid->h0[a] * n[a], r = std::nearbyint(x);
        if (!(fabs(x - r) < 1e-6) || fabs(r) > 1e8)
            return say(err, errlen, DS_ERR_UNSUPPORTED, "grid axis %d: h0 * n is not an integer", a);
        g0[a] = (int)r;
        cnt[a] = (int)grid->count[a];
    }
    const GridMap gm = grid_map(g, g0, cnt);
    double A[9], B[9];
    lattice_matrices(lattice, A, B);
    if (!(A[8] > 0) || !std::isfinite(B[0])) return say(err, errlen, DS_ERR_ARG, "degenerate lattice");

    // sites sorted by z = r3 mod 1 (one form-factor class: constant), groups of equal z
    std::vector<int> site_of(nsite);
    for (int i = 0; i < nsite; ++i) site_of[i] = i;
    auto zf = [&](int s) { return frac_xyz[3 * s + 2] - floor(frac_xyz[3 * s + 2]); };
    std::stable_sort(site_of.begin(), site_of.end(), [&](int x, int y) { return zf(x) < zf(y); });
    RecombParams<float> p;
    memset(&p, 0, sizeof(p));
    SiteGroups &G = p.grp;
    for (int i = 0; i < nsite; ++i) {
        if (i == 0 || zf(site_of[i]) != zf(site_of[i - 1])) G.grp_site[G.ngrp++] = site_of[i];
        G.grp_end[G.ngrp - 1] = i + 1;
    }
    G.cls_grp_end[0] = G.ngrp;
    for (int c = 1; c < MAX_FF_CLASSES; ++c) G.cls_grp_end[c] = -1;
    p.ff.ncls = 1;
    p.ff.cls_kind[0] = DS_FF_CONST;
    gaussian_sum_form(p.ff, 0, DS_FF_CONST, nullptr);
    p.ff.cls_end[0] = nsite;
    for (int c = 1; c < MAX_FF_CLASSES; ++c) p.ff.cls_end[c] = -1;

    // scratch layout
    const int nmax = std::max(n1, std::max(n2, n3));
    const int nHmax = std::max(gm.nH[0], std::max(gm.nH[1], gm.nH[2]));
    const int nf = nmodels * nsite;
    const int fb = std::min(nf, 64);
    size_t off = 0;
    const size_t o_tw = off;
    off = align256(off + sizeof(C) * (n1 + n2 + n3));
    const size_t o_phk = off;
    off = align256(off + sizeof(C) * nsite * 3 * nmax);
    const size_t o_phH = off;
    off = align256(off + sizeof(C) * nsite * 3 * nHmax);
    const size_t o_sites = off;
    off = align256(off + sizeof(double) * 3 * nsite);
    const size_t o_site_of = off;
    off = align256(off + sizeof(int) * nsite);
    const size_t o_scat = off;
    off = align256(off + sizeof(float) * nsite);
    const size_t o_mean = off;
    off = align256(off + sizeof(double) * nsite);
    const size_t o_spec = off;
    off = align256(off + sizeof(C) * (size_t)nf * g.ncell_h);
    const size_t o_work = off;
    off = align256(off + sizeof(C) * (size_t)fb * g.ncell_h);
    if (off > DS_NOALLOC_SCRATCH_BYTES)
        return say(err, errlen, DS_ERR_ADMISSION,
                   "request needs %zu bytes of scratch; the static scratch of this entry point holds %u bytes", off,
                   (unsigned)DS_NOALLOC_SCRATCH_BYTES);

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaSetDevice(dev) != cudaSuccess)
        return say(err, errlen, DS_ERR_CUDA, "no current CUDA device");
    unsigned char *base = nullptr;
    ds_status rc = scratch_address(dev, &base, err, errlen);
    if (rc != DS_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;

    C *tw = (C *)(base + o_tw);
    C *W[3] = {tw, tw + n1, tw + n1 + n2};
    double *d_sites = (double *)(base + o_sites);
    int *d_site_of = (int *)(base + o_site_of);
    float *d_scat = (float *)(base + o_scat);
    double *d_mean = (double *)(base + o_mean);
    SiteInputs in;
    memset(&in, 0, sizeof(in));
    in.nsite = nsite;
    in.has_mean = mean_occ != nullptr;
    for (int i = 0; i < nsite; ++i) {
        for (int a = 0; a < 3; ++a) in.frac[3 * i + a] = frac_xyz[3 * i + a];
        in.site_of[i] = site_of[i];
        in.scat[i] = scat_len ? (float)scat_len[i] : 1.0f;
        in.mean[i] = mean_occ ? mean_occ[i] : 0.0;
    }
    k_noalloc_sites<<<1, kMaxSites, 0, st>>>(in, d_sites, d_site_of, d_scat, d_mean);
    count_launches(1);
    for (int a = 0; a < 3; ++a) make_twiddles<float>(n[a], W[a], st);

    p.g = g;
    p.gm = gm;
    p.nsite = nsite;
    p.nmodels = nmodels;
    p.ncomp = 1;
    p.diffuse = mode == DS_DIFFUSE;
    set_reciprocal(p, B, g.n);
    p.norm = (float)(1.0 / ((double)nmodels * nsite * g.ncell));
    p.nmax = nmax;
    p.nHmax = nHmax;
    p.phk = (C *)(base + o_phk);
    p.phH = (C *)(base + o_phH);
    p.site_of = d_site_of;
    p.sites = d_sites;
    p.scat = d_scat;
    p.out = out_dev;
    make_site_tables<float>(g, gm, nsite, d_sites, (C *)(base + o_phk), (C *)(base + o_phH), nmax, nHmax, st);

    FieldSource src;
    memset(&src, 0, sizeof(src));
    src.kind = SRC_OCC;
    src.nsite = nsite;
    src.nf_per_model = nsite;
    src.diffuse = p.diffuse;
    src.occ = occ_dev;
    src.mean = d_mean;
    if (p.diffuse && !mean_occ) site_means_occ(nmodels, nsite, g.ncell, occ_dev, d_mean, st);
    C *spec = (C *)(base + o_spec);
    C *work = (C *)(base + o_work);
    for (int f0 = 0; f0 < nf; f0 += fb)
        fft_real_fields<float>(g, src, f0, std::min(fb, nf - f0), work, spec, W[0], W[1], W[2], st);
    p.spec = spec;
    for (int m = 0; m < nmodels; ++m) {
        p.model = m;
        p.accumulate = m > 0;
        recombine_cm<float>(p, st);
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return say(err, errlen, DS_ERR_CUDA, "launch failed: %s", cudaGetErrorString(e));
    return DS_OK;
}
