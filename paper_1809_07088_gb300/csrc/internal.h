// Internal interfaces between the C-ABI runtime (api.cu) and the kernel translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "ds_common.cuh"
#include "fft_lines.cuh"

namespace ds {

// kernels launched by the library (read and reset by ds_profile_report)
void count_launches(int n);

// supercell grid and its FFT plan
struct Geometry {
    int n[3];       // n1, n2, n3 (unit cells per axis)
    int n3h;        // n3 / 2 + 1: stored half of the last axis (real input)
    int ncell;      // n1 n2 n3
    int ncell_h;    // n1 n2 n3h
    AxisPlan ax[3];
};

// index of the stored half-spectrum element holding X(k) (conj = 1 when X(k) = conj X(-k))
__host__ __device__ __forceinline__ int half_index(const Geometry &g, int k1, int k2, int k3, int &conj) {
    if (k3 < g.n3h) {
        conj = 0;
        return (k1 * g.n[1] + k2) * g.n3h + k3;
    }
    conj = 1;
    const int m1 = (g.n[0] - k1) % g.n[0], m2 = (g.n[1] - k2) % g.n[1], m3 = (g.n[2] - k3) % g.n[2];
    return (m1 * g.n[1] + m2) * g.n3h + m3;
}

// what a real FFT field is made of
enum SourceKind { SRC_OCC = 0, SRC_SPIN = 1, SRC_DISP = 2, SRC_REAL = 3 };

struct FieldSource {
    int kind;
    int nsite;
    int nf_per_model;   // fields per supercell (nsite, 3 nsite or nsite T)
    int diffuse;        // subtract the site means (occupancy / moment)
    const uint8_t *occ; // [model][site][cell]
    const float *vec3;  // spins [model][site][cell][3]
    const double *mean; // occupancy mean [site] or moment mean [site][3]
    const void *pw;     // displacive powers (T) [model][site][3][P+1][cell]: (u Qs)^e / e!
    const int4 *terms;  // displacive monomials (a, b, c, n), lexicographic
    int T, P;           // number of monomials, order
    const void *real_buf; // SRC_REAL: [field][cell] (T)
};

// output grid in supercell indices G_alpha = g0_alpha + i_alpha, split into zones H
struct GridMap {
    int g0[3];
    int cnt[3];
    int Hmin[3];
    int nH[3];
};

template <typename T> struct FormFactors {
    int ncls;                       // classes = contiguous ranges of the sorted sites
    int cls_end[MAX_FF_CLASSES];    // exclusive end (sorted position)
    int cls_kind[MAX_FF_CLASSES];
    T cls_coef[MAX_FF_CLASSES][9];
    // the same form factors as sums of Gaussians in |Q|^2: f = gc + sum_{i < ng} ga_i 2^(gb_i |Q|^2)
    int cls_ng[MAX_FF_CLASSES];
    T cls_ga[MAX_FF_CLASSES][4], cls_gb[MAX_FF_CLASSES][4], cls_gc[MAX_FF_CLASSES];
};

// fills the Gaussian-sum form of class c from its kind and coefficients (s = |Q| / 4 pi)
template <typename T> inline void gaussian_sum_form(FormFactors<T> &ff, int c, int kind, const double *coef) {
    const double to_q2 = 1.4426950408889634 / (16.0 * 9.869604401089358);  // log2(e) / (4 pi)^2
    double a[4] = {0, 0, 0, 0}, b[4] = {0, 0, 0, 0}, c0 = 1.0;
    int ng = 0;
    if (kind == 1) {  // sum_i a_i exp(-b_i s^2) + c
        for (int i = 0; i < 4; ++i) a[i] = coef[i], b[i] = coef[4 + i];
        ng = 4;
        c0 = coef[8];
    } else if (kind == 2) {  // A exp(-a s^2) + B exp(-b s^2) + C exp(-c s^2) + D
        a[0] = coef[0], b[0] = coef[1], a[1] = coef[2], b[1] = coef[3];
        ng = 2;
        if (coef[4] != 0.0) a[2] = coef[4], b[2] = coef[5], ng = 3;
        c0 = coef[6];
    }
    ff.cls_ng[c] = ng;
    for (int i = 0; i < 4; ++i) {
        ff.cls_ga[c][i] = (T)a[i];
        ff.cls_gb[c][i] = (T)(-b[i] * to_q2);
    }
    ff.cls_gc[c] = (T)c0;
}

// sites sorted by (form-factor class, z = r_mu,3 mod 1); a group = sites of one class sharing z,
// so that exp(2 pi i H3 z) is common to the group
struct SiteGroups {
    int ngrp;
    int grp_end[MAX_SITES];            // exclusive end of each group (sorted positions)
    int grp_site[MAX_SITES];           // one site of each group (its z is the group's)
    int cls_grp_end[MAX_FF_CLASSES];   // exclusive end of each form-factor class (group index)
};

// plan of the sum-factorised Taylor recombination (taylor_sf.cu): the monomial exponents a are
// processed in groups (shared-memory budget), each group's (a, b) pairs listed in a balanced order
constexpr int SF_MAX_GROUPS = 24;
struct SFPlan {
    int zr;                            // register width: zones per axis of a CTA's box (<= zr)
    int ngroups;
    int a0[SF_MAX_GROUPS + 1];         // group g holds a in [a0[g], a0[g+1])
    int ibeg[SF_MAX_GROUPS + 1];       // its slots in `items`: [ibeg[g], ibeg[g+1])
    int xpad;                          // row stride of the per-group partial sums X[h3][item]
    int ymax;                          // largest group (a values)
    size_t smem;                       // dynamic shared memory of one CTA
    int nthr;                          // threads per CTA (128, 256 or 512: 16 warps per SM)
    const int4 *items;                 // slots: (a, b, t0, xi), a < 0 = empty slot
};

template <typename T> struct RecombParams {
    Geometry g;
    GridMap gm;
    int nsite, nmodels, model;          // model: which supercell this launch handles
    int ncomp;                          // 1 (occupancy / displacive) or 3 (magnetic)
    int nT;                             // monomials per site (displacive)
    int accumulate;                     // add into out instead of overwriting
    int diffuse;
    const c_t<T> *spec;                 // [model][site][ncomp or T][ncell_h]
    const c_t<T> *phk;                  // [site][3][nmax]   exp(2 pi i k_a r_a / n_a)
    const c_t<T> *phH;                  // [site][3][nHmax]  exp(2 pi i H_a r_a)
    int nmax, nHmax;
    const int *site_of;                 // sorted position -> site
    const double *sites;                // fractional site coordinates [site][3]
    const T *scat;                      // b per site
    FormFactors<T> ff;
    SiteGroups grp;
    double recip[9];                    // a*, b*, c* rows (1/A)
    T qstep[9];                         // a*/n1, b*/n2, c*/n3 rows: Q = sum_a G_a qstep_a
    double gscale[3];                   // displacive: coefficients use x_a = g_a / gscale_a, g_a = G_a / n_a
    const c_t<T> *phHx;                 // displacive: exp(2 pi i H_a r_a) [site][3][nHx] over the zones of
    int Hminx[3], nHx;                  //   the grid and of its negation (Friedel mates), from zone Hminx
    T norm;                             // 1/(nmodels N), times C for magnetic
    const int *ops;                     // displacive coefficient update codes per monomial
    const int4 *terms;                  // displacive monomials (a, b, c, n)
    const int *pzone;                   // optional: Taylor order of each zone [nH1][nH2][nH3]
    const int *sub_map;                 // order-p sub-simplex in lexicographic order -> global monomial
    const int *sub_ops;                 // its coefficient update codes
    const int *sub_off;                 // offset of order p in sub_map / sub_ops
    const c_t<T> *bragg;                // displacive DIFFUSE: <F(H)> per zone [nH1][nH2][nH3]
    T *out;                             // [cnt1][cnt2][cnt3]
    c_t<T> *Fout;                       // optional: F per voxel [model][voxel][ncomp] (adjoint)
    int force_plain;                    // use the per-site (ungrouped) recombination
    int dres[3];                        // residue classes of zones per axis (0: per-zone kernels)
    const T *dw;                        // optional: Debye-Waller factor T_mu(G) [site][voxel] (magnetic)
    SFPlan sf;                          // displacive, sum-factorised recombination
    int *err;
};

// reciprocal rows (FP64, Cartesian 1/A) and their per-supercell-index steps in the working type
template <typename T> inline void set_reciprocal(RecombParams<T> &p, const double recip[9], const int n[3]) {
    for (int i = 0; i < 9; ++i) {
        p.recip[i] = recip[i];
        p.qstep[i] = (T)(recip[i] / n[i / 3]);
    }
}

// ---- launchers (fft.cu) --------------------------------------------------------------------
template <typename T> void make_twiddles(int n, c_t<T> *W, cudaStream_t s);
template <typename T>
void fft_real_fields(const Geometry &g, const FieldSource &src, int f0, int nf, c_t<T> *work,
                     c_t<T> *spec, const c_t<T> *W1, const c_t<T> *W2, const c_t<T> *W3, cudaStream_t s);
size_t fft_work_bytes(const Geometry &g, int nf, size_t elem);

// ---- launchers (recomb.cu) -----------------------------------------------------------------
template <typename T>
void make_site_tables(const Geometry &g, const GridMap &gm, int nsite, const double *sites_dev,
                      c_t<T> *phk, c_t<T> *phH, int nmax, int nHmax, cudaStream_t s);
// pw[m][s][a][e][cell] = (gscale_a u~_a)^e / e!, u~_a = b*_a . u (recip rows b*_a, Cartesian)
template <typename T>
void make_powers(const Geometry &g, int nmodels, int nsite, int P, const double recip[9], const double gscale[3],
                 const float *disp, T *pw, cudaStream_t s);
void site_means_occ(int nmodels, int nsite, int ncell, const uint8_t *occ, double *mean, cudaStream_t s);
void site_means_spin(int nmodels, int nsite, int ncell, const float *spins, double *mean, cudaStream_t s);
struct Corners {
    double v[24];  // 8 Cartesian Q vectors
};
// out (device, 9 doubles): max_j |Q_c . u_j| for the 8 corners, then max_j |u_j|
void corner_xmax(int natom, const float *disp, const Corners &corners, double *out, cudaStream_t s);
template <typename T> void recombine_cm(const RecombParams<T> &p, cudaStream_t s);
// recomb_res.cu: the residue-class kernel when p.dres is set; false when it does not apply
template <typename T> bool recombine_cm_residues(const RecombParams<T> &p, cudaStream_t s);
// recomb_rows.cu: the residue-class table + whole-row writer (one form-factor class); false when it
// does not apply
template <typename T> bool recombine_rows(const RecombParams<T> &p, cudaStream_t s);
template <typename T> void recombine_disp(const RecombParams<T> &p, cudaStream_t s);
// taylor_sf.cu: the displacive recombination by sum factorisation over the zones of each k (one
// Taylor order for the grid); false when it does not apply (zone orders, zone boxes too large)
template <typename T> void recombine_disp_sf(const RecombParams<T> &p, cudaStream_t s);
// host plan of that kernel (false: zone boxes wider than it handles, or, unless forced, more work
// than the per-voxel recombination); `items` is the slot table to upload, its device address then
// goes into plan.items
// threads per CTA (128, 256 or 512) keeping 16 warps on an SM for a dynamic shared-memory footprint
int sf_threads_for(size_t smem);
bool taylor_sf_plan(const Geometry &g, const GridMap &gm, int P, int nsite, size_t celem, bool force, SFPlan &plan,
                    std::vector<int4> &items);
template <typename T>
void displacive_bragg(const RecombParams<T> &p, const int4 *terms, c_t<T> *avg0, c_t<T> *bragg, cudaStream_t s);

}  // namespace ds
