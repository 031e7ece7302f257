// Internal interfaces between the C-ABI runtime (api.cu) and the kernel translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

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
};

// sites sorted by (form-factor class, z = r_mu,3 mod 1); a group = sites of one class sharing z,
// so that exp(2 pi i H3 z) is common to the group
struct SiteGroups {
    int ngrp;
    int grp_end[MAX_SITES];            // exclusive end of each group (sorted positions)
    int grp_site[MAX_SITES];           // one site of each group (its z is the group's)
    int cls_grp_end[MAX_FF_CLASSES];   // exclusive end of each form-factor class (group index)
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
    double qscale;                      // displacive: coefficient uses Q / qscale
    T norm;                             // 1/(nmodels N), times C for magnetic
    const int *ops;                     // displacive coefficient update codes per monomial
    const int4 *terms;                  // displacive monomials (a, b, c, n)
    const c_t<T> *bragg;                // displacive DIFFUSE: <F(H)> per zone [nH1][nH2][nH3]
    T *out;                             // [cnt1][cnt2][cnt3]
    c_t<T> *Fout;                       // optional: F per voxel [model][voxel][ncomp] (adjoint)
    int force_plain;                    // use the per-site (ungrouped) recombination
    int *err;
};

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
template <typename T>
void make_powers(const Geometry &g, int nmodels, int nsite, int P, double qscale, const float *disp,
                 T *pw, cudaStream_t s);
void site_means_occ(int nmodels, int nsite, int ncell, const uint8_t *occ, double *mean, cudaStream_t s);
void site_means_spin(int nmodels, int nsite, int ncell, const float *spins, double *mean, cudaStream_t s);
struct Corners {
    double v[24];  // 8 Cartesian Q vectors
};
void corner_xmax(int natom, const float *disp, const Corners &corners, double *out /*dev [8]*/, cudaStream_t s);
template <typename T> void recombine_cm(const RecombParams<T> &p, cudaStream_t s);
template <typename T> void recombine_disp(const RecombParams<T> &p, cudaStream_t s);
template <typename T>
void displacive_bragg(const RecombParams<T> &p, const int4 *terms, c_t<T> *avg0, c_t<T> *bragg, cudaStream_t s);

}  // namespace ds
