// Host-side state behind the opaque C handles, shared by api.cu, serving.cu, subbox.cu and
// adjoint.cu.
#pragma once

#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <set>
#include <string>
#include <thread>
#include <vector>

#include "../../include/ds.h"
#include "internal.h"

struct ServeJob;

struct ds_model {
    ds_ctx *ctx = nullptr;
    double lat[6] = {0};
    double A[9] = {0}, recip[9] = {0};
    bool has_lattice = false;
    int nsite = 0;
    std::vector<double> sites, scat, ffcoef;
    std::vector<int> ffkind;
    int n[3] = {0, 0, 0};
    int nmodels = 0;
    bool has_cells = false;
    uint8_t *d_occ = nullptr;
    float *d_spins = nullptr;
    float *d_disp = nullptr;
    double *d_sites = nullptr;
    bool has_occ = false, has_spins = false, has_disp = false;
    bool user_mean = false;
    std::vector<double> mean_occ;
    double *d_user_mean = nullptr;
    // per-model constants of the launch sequence, built once by set_sites / set_supercell
    bool ff_ok = false;
    std::vector<int> site_of;             // sorted position -> site (form-factor classes contiguous)
    ds::FormFactors<float> ff32;
    ds::FormFactors<double> ff64;
    ds::SiteGroups groups;
    int period[3] = {0, 0, 0};            // smallest d <= 64 with d r_mu,a integral for all sites (0: none)
    // per-site means of the uploaded data (Eq. occ: c_mu; mean moments), computed at upload
    double *d_mean_occ = nullptr;         // [site]
    double *d_mean_spin = nullptr;        // [site][3]
    cudaEvent_t ready = nullptr;          // recorded after every upload; every request stream waits on it
    // site phase tables per grid, built by the first request that needs them
    struct SiteTables {
        void *phk = nullptr, *phH = nullptr;
        cudaEvent_t done = nullptr;       // recorded after the tables' kernel on the building stream
    };
    std::map<std::vector<int>, SiteTables> site_tables;  // (precision, Hmin, nH) -> tables
    std::mutex cache_mu;                  // guards the caches of this model (serving worker and callers)
    int *d_site_of = nullptr;
    float *d_scat32 = nullptr;
    double *d_scat64 = nullptr;
    ds::c_t<float> *d_tw32[3] = {nullptr, nullptr, nullptr};
    ds::c_t<double> *d_tw64[3] = {nullptr, nullptr, nullptr};
    std::map<int, std::pair<int4 *, int *>> taylor_tables;   // order P -> (terms, ops) on device
    std::map<int, int *> sub_tables;                          // order P -> sub-simplex tables (map, ops, off)
};

struct ProfRecord {
    std::string name;
    cudaEvent_t e0, e1;
};

struct ds_ctx {
    int device = 0;
    // tracing
    bool prof_on = false;
    std::mutex prof_mu;
    std::vector<ProfRecord> prof;
    std::vector<cudaEvent_t> event_pool;   // reused by the tracing scopes
    size_t budget = 0;
    std::mutex err_mu;
    std::string err;
    cudaStream_t stream = nullptr;
    std::set<ds_model *> models;
    // serving (serving.cu)
    std::mutex mu;
    std::condition_variable cv;
    std::thread worker;
    bool worker_started = false;
    bool stop = false;
    bool paused = false;
    uint64_t next_ticket = 1;
    std::deque<ServeJob *> queue;
    std::map<uint64_t, ServeJob *> jobs;
    size_t inflight_bytes = 0;
    std::vector<cudaStream_t> serve_streams;   // the first half at the highest stream priority
    std::vector<int> stream_jobs;              // jobs in flight per serving stream
    std::deque<double> recent_cost;            // costs of the latest admitted jobs (priority split)
    double *plan_host = nullptr;               // pinned slots for the x_max read-backs of planning
    std::vector<int> plan_free;                // free slots of plan_host
    cudaStream_t plan_stream = nullptr;        // x_max reductions of served displacive requests
};

ds_status ds_fail(ds_ctx *ctx, ds_status st, const char *fmt, ...);

// brackets one kernel stage with events when profiling is on
struct ProfScope {
    ProfScope(ds_ctx *ctx, const char *name, cudaStream_t s);
    ~ProfScope();
    ds_ctx *ctx;
    cudaStream_t s;
    ProfRecord rec;
    bool on;
};

// stream-ordered scratch of one request
struct Scratch {
    explicit Scratch(cudaStream_t s) : stream(s) {}
    ~Scratch();
    void *get(size_t bytes);
    void release();
    cudaStream_t stream;
    std::vector<void *> ptrs;
    size_t total = 0;
    bool failed = false;
};

// what the adjoint reuses from the forward plan
template <typename T> struct ForwardKeep {
    ds::RecombParams<T> p;
    ds::Geometry g;
    ds::FieldSource src;
    const ds::c_t<T> *W[3];
    const int4 *terms = nullptr;
    const T *pw = nullptr;
    ds::c_t<T> *Fout = nullptr;   // requested: F per voxel is written here
};

void lattice_matrices(const double lat[6], double A[9], double B[9]);
bool make_geometry(const int n[3], ds::Geometry &g);
ds::GridMap grid_map(const ds::Geometry &g, const int g0[3], const int cnt[3]);
ds_status grid_indices(ds_ctx *ctx, const ds_model *M, const ds_qgrid *q, int g0[3], int cnt[3]);
ds_status check_request(ds_model *M, const ds_qgrid *q, const ds_opts *o);
void monomial_tables(int P, std::vector<int4> &terms, std::vector<int> &ops);
int taylor_order_for(double xmax, double eps);
void box_corners(const ds_model *M, const int g0[3], const int cnt[3], double corners[24]);

// a Taylor order resolved ahead of launch (serving plans on the submitting thread)
struct TaylorHint {
    int P;
    double xmax, umax;
};

// the forward calculation into a device buffer on stream st, scratch from ws
template <typename T>
ds_status plan_and_run(ds_model *M, const ds_qgrid *q, const ds_opts *o, T *d_out, cudaStream_t st, Scratch &ws,
                       ds_result_info *info, ForwardKeep<T> *keep, const TaylorHint *hint = nullptr);
// all kernels of one request into a device volume, no synchronisation (smoothing included)
template <typename T>
ds_status enqueue_request(ds_model *M, const ds_qgrid *q, const ds_opts *o, T *d_out, cudaStream_t st, Scratch &ws,
                          ds_result_info *info, const TaylorHint *hint = nullptr);
ds_status resolve_taylor_order(ds_model *M, const ds_qgrid *q, const ds_opts *o, cudaStream_t st, Scratch &ws, int *P,
                               double *xmax, double *umax = nullptr);
ds_status queue_corner_xmax(ds_model *M, const ds_qgrid *q, const ds_opts *o, cudaStream_t st, Scratch &ws,
                            double *host_out);
ds_status taylor_order_from_corners(ds_ctx *ctx, const ds_opts *o, const double hx[9], int *P, double *xmax,
                                    double *umax);
size_t request_footprint(const ds_model *M, const ds_qgrid *q, const ds_opts *o, int P);
bool residue_classes(const ds_model *M, const ds::GridMap &gm, int dres[3]);
// Lanczos resampling with the separable or the spherical cutoff (api.cu)
bool lanczos_like(const ds_opts *o);
double sphere_cutoff_radius(const ds_model *M, int m, int mprime);
double sphere_profile(double x);
void sphere_stencil_weights(const ds_model *M, int m, int mprime, int h, std::vector<double> &w);
// T_mu(G) of Eq. dw on the grid g0 + [0, cnt) of supercell indices, [site][voxel] (subbox_dft.cu)
template <typename T> void debye_waller_grid(const ds_model *M, const int g0[3], const int cnt[3], T *out, cudaStream_t st);
// sub-box averaging (subbox.cu)
template <typename T>
ds_status subbox_run(ds_model *M, const ds_qgrid *q, const ds_opts *o, T *d_out, cudaStream_t st, Scratch &ws,
                     ds_result_info *info);
// serving (serving.cu)
void serving_shutdown(ds_ctx *ctx);
