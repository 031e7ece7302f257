/*
 * CPU FP64 oracle, part 1: the direct (single-sum) structure factor.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path links, loads or calls this file; it
 * is compiled by oracle/build.py and called from the test-suite, from the smoke check and from
 * the CPU-baseline leg of the benchmark.
 *
 * It evaluates the definition of the structure factor, Eq. (sf) of Section II,
 *
 *     F(Q) = sum_j  b_j f_j(|Q|)  exp(i Q . r_j)
 *
 * with the atom positions decomposed as r = R + r_mu + u (Eq. r_vec, Section III A): the
 * lattice part R + r_mu is passed in fractional unit-cell coordinates, so that
 * Q . (R + r_mu) = 2 pi (h x + k y + l z) exactly, and the displacement u in Cartesian
 * Angstrom, so that its phase is Q_cart . u.  Up to three real amplitudes per atom (ncomp) are
 * summed with the same phase: ncomp = 1 for nuclear scattering (amplitude b * occupancy),
 * ncomp = 3 for the magnetic structure factor vector (amplitude = moment components, Eq.
 * mag_sf of Section III D).
 *
 * Form factors (the paper leaves their functional form open): kind 0 = 1 (constant, the
 * scattering length alone), kind 1 = sum_{i=1..4} a_i exp(-b_i s^2) + c, kind 2 = magnetic
 * <j0> = A exp(-a s^2) + B exp(-b s^2) + C exp(-c s^2) + D, with s = |Q| / (4 pi).
 * Coefficient layout, 9 doubles per site: kind 1 (a1 a2 a3 a4 b1 b2 b3 b4 c); kind 2
 * (A a B b C c D - -).
 *
 * Plain loops, FP64 round-to-nearest, OpenMP over Q points only.
 */
#include <math.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define TWO_PI 6.283185307179586476925286766559
#define FOUR_PI 12.566370614359172953850573533118

static double oracle_form_factor(int kind, const double *c, double qnorm)
{
    double s2 = (qnorm / FOUR_PI) * (qnorm / FOUR_PI);
    if (kind == 1)
        return c[0] * exp(-c[4] * s2) + c[1] * exp(-c[5] * s2) + c[2] * exp(-c[6] * s2) +
               c[3] * exp(-c[7] * s2) + c[8];
    if (kind == 2)
        return c[0] * exp(-c[1] * s2) + c[2] * exp(-c[3] * s2) + c[4] * exp(-c[5] * s2) + c[6];
    return 1.0;
}

/* Returns the number of OpenMP threads used (1 without OpenMP). */
int oracle_threads(void)
{
#ifdef _OPENMP
    int n = 1;
#pragma omp parallel
    {
#pragma omp single
        n = omp_get_num_threads();
    }
    return n;
#else
    return 1;
#endif
}

/*
 * natom          number of atoms
 * frac[natom*3]  R + r_mu in fractional unit-cell coordinates
 * ucart          [natom*3] Cartesian displacements (A), or NULL for none
 * ncomp, amp     [natom*ncomp] real amplitudes
 * site[natom]    site index of each atom (selects its form factor)
 * nsite, ffkind[nsite], ffcoef[nsite*9]
 * recip[9]       rows a*, b*, c* (Cartesian, 1/A, including the 2 pi)
 * nq, hkl[nq*3]  wavevectors in r.l.u.
 * F[nq*ncomp*2]  output, (re, im) pairs
 */
void oracle_structure_factor(long natom, const double *frac, const double *ucart, int ncomp,
                             const double *amp, const int *site, int nsite, const int *ffkind,
                             const double *ffcoef, const double *recip, long nq,
                             const double *hkl, double *F)
{
#pragma omp parallel
    {
        double *ff = (double *)malloc(sizeof(double) * (size_t)(nsite > 0 ? nsite : 1));
#pragma omp for schedule(dynamic, 16)
        for (long q = 0; q < nq; ++q) {
            const double h = hkl[3 * q + 0], k = hkl[3 * q + 1], l = hkl[3 * q + 2];
            double Q[3];
            for (int a = 0; a < 3; ++a)
                Q[a] = h * recip[0 * 3 + a] + k * recip[1 * 3 + a] + l * recip[2 * 3 + a];
            const double qn = sqrt(Q[0] * Q[0] + Q[1] * Q[1] + Q[2] * Q[2]);
            for (int s = 0; s < nsite; ++s)
                ff[s] = oracle_form_factor(ffkind[s], ffcoef + 9 * s, qn);
            double acc[3][2] = {{0, 0}, {0, 0}, {0, 0}};
            for (long j = 0; j < natom; ++j) {
                double t = h * frac[3 * j + 0] + k * frac[3 * j + 1] + l * frac[3 * j + 2];
                t -= floor(t); /* exp(2 pi i t) depends on t mod 1 only */
                double phase = TWO_PI * t;
                if (ucart)
                    phase += Q[0] * ucart[3 * j + 0] + Q[1] * ucart[3 * j + 1] +
                             Q[2] * ucart[3 * j + 2];
                const double cr = cos(phase), ci = sin(phase);
                const double f = ff[site[j]];
                for (int c = 0; c < ncomp; ++c) {
                    const double a = amp[(long)ncomp * j + c] * f;
                    acc[c][0] += a * cr;
                    acc[c][1] += a * ci;
                }
            }
            for (int c = 0; c < ncomp; ++c) {
                F[2 * ((long)ncomp * q + c) + 0] = acc[c][0];
                F[2 * ((long)ncomp * q + c) + 1] = acc[c][1];
            }
        }
        free(ff);
    }
}
