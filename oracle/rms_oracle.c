/*
 * FP64 CPU oracle for RM synthesis (Sridhar, Heald & van der Hulst,
 * "cuFFS: A GPU-accelerated code for Fast Faraday Rotation Measure Synthesis").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain definition that the
 * GPU library is checked against.  Only tests/, __graft_entry__.smoke() and
 * bench.py's CPU-baseline leg may load it.  It shares no code, header, table
 * or constant with the CUDA library under paper_1810_06250_gb300/, and it
 * never reads anything the CUDA library produced.
 *
 * Every sum is a plain double-precision loop in the order the paper states:
 * for one line of sight, the outer loop runs over channels and the inner loop
 * over all Faraday depths (Sec. 3, the Brentjens CPU strategy).  cos/sin are
 * called on the full, unreduced double argument; glibc reduces it exactly.
 *
 * Readings of the paper taken here:
 *  - lambda_0^2 is the weighted mean of lambda_i^2 over the weights
 *    (Sec. 2.2 says "mean of lambda_i^2"; weighted = plain mean for uniform
 *    weights and makes dR/dphi(0) = 0).
 *  - The weights w_i multiply P_i in the real (Q, U) form too (Eq. Fsum uses
 *    P~ = W P; the printed real form omits w_i).
 *  - Channels with w_i == 0 are skipped entirely, so NaN/Inf data in flagged
 *    channels has no effect (Sec. 2.1: W is zero where P was not measured).
 *  - Exponent sign e^{-2 i phi (lambda^2 - lambda_0^2)} (Eq. Fsum), which is
 *    the same as Q~ = K sum (Q cos + U sin), U~ = K sum (U cos - Q sin)
 *    (Eqs. qPhi, uPhi).
 *
 * Build: gcc -O2 -fopenmp -fPIC -shared rms_oracle.c -lm -o liboracle.so
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Speed of light in m/s (exact, SI definition). */
static const double ORACLE_C_LIGHT = 299792458.0;

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/*
 * Plan constants, Sec. 2.2.
 *   lambda_i^2 = (c / nu_i)^2 when kind == 1 (axis in Hz), else axis itself.
 *   K = (sum_i w_i)^-1                                 (Eq. Ksum)
 *   lambda_0^2 = sum_i w_i lambda_i^2 / sum_i w_i      (weighted mean, see above)
 * weights == NULL means w_i = 1 for every channel.
 * Returns 0 on success, -1 when a weight is negative or non-finite or the sum
 * of weights is not positive, -2 when an axis value is not finite (or a
 * frequency is not positive).
 */
int oracle_plan(const double *axis, int32_t nchan, int32_t kind, const double *weights,
                double *lambda2, double *K, double *lambda0sq)
{
    double sw = 0.0, swl = 0.0;
    for (int32_t i = 0; i < nchan; ++i) {
        double a = axis[i];
        if (!isfinite(a)) return -2;
        if (kind == 1) {
            if (!(a > 0.0)) return -2;
            double lam = ORACLE_C_LIGHT / a;
            lambda2[i] = lam * lam;
        } else {
            lambda2[i] = a;
        }
        double w = weights ? weights[i] : 1.0;
        if (!isfinite(w) || w < 0.0) return -1;
        sw += w;
        swl += w * lambda2[i];
    }
    if (!(sw > 0.0)) return -1;
    *K = 1.0 / sw;
    *lambda0sq = swl / sw;
    return 0;
}

/*
 * RM synthesis, Eq. Fsum:  F(phi_k) = K sum_i w_i P_i exp(-2 i phi_k (lambda_i^2 - lambda_0^2))
 * with P_i = Q_i + i U_i.
 *   Q, U : [nlos][nchan] row-major (line-of-sight major), double
 *   F    : [nlos][nphi][2] (re, im), overwritten
 * One thread per line of sight (OpenMP); inside, channel-outer / phi-inner.
 */
void oracle_synth(int64_t nlos, int32_t nchan, const double *Q, const double *U,
                  const double *lambda2, const double *weights, double lambda0sq, double K,
                  const double *phi, int32_t nphi, double *F)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t l = 0; l < nlos; ++l) {
        double *Fl = F + (size_t)l * (size_t)nphi * 2;
        for (int32_t k = 0; k < nphi; ++k) { Fl[2 * k] = 0.0; Fl[2 * k + 1] = 0.0; }
        const double *Ql = Q + (size_t)l * (size_t)nchan;
        const double *Ul = U + (size_t)l * (size_t)nchan;
        for (int32_t i = 0; i < nchan; ++i) {
            double w = weights ? weights[i] : 1.0;
            if (w == 0.0) continue;               /* flagged channel: W(lambda_i^2) = 0 */
            double q = w * Ql[i], u = w * Ul[i];  /* P~_i = w_i P_i */
            double d = lambda2[i] - lambda0sq;
            for (int32_t k = 0; k < nphi; ++k) {
                double theta = 2.0 * phi[k] * d;
                double c = cos(theta), s = sin(theta);
                /* (q + i u)(c - i s) = (q c + u s) + i (u c - q s) */
                Fl[2 * k] += q * c + u * s;
                Fl[2 * k + 1] += u * c - q * s;
            }
        }
        for (int32_t k = 0; k < nphi; ++k) { Fl[2 * k] *= K; Fl[2 * k + 1] *= K; }
    }
}

/*
 * RMSF, Eq. Rsum:  R(phi_k) = K sum_i w_i exp(-2 i phi_k (lambda_i^2 - lambda_0^2)).
 *   R : [nphi][2] (re, im)
 */
void oracle_rmsf(int32_t nchan, const double *lambda2, const double *weights, double lambda0sq,
                 double K, const double *phi, int32_t nphi, double *R)
{
    for (int32_t k = 0; k < nphi; ++k) { R[2 * k] = 0.0; R[2 * k + 1] = 0.0; }
    for (int32_t i = 0; i < nchan; ++i) {
        double w = weights ? weights[i] : 1.0;
        if (w == 0.0) continue;
        double d = lambda2[i] - lambda0sq;
        for (int32_t k = 0; k < nphi; ++k) {
            double theta = 2.0 * phi[k] * d;
            R[2 * k] += w * cos(theta);
            R[2 * k + 1] -= w * sin(theta);
        }
    }
    for (int32_t k = 0; k < nphi; ++k) { R[2 * k] *= K; R[2 * k + 1] *= K; }
}

/*
 * Peak of |F| per line of sight (Sec. 2.2: phi_peak is where |F~(phi)| is
 * largest, |F~| = sqrt(Q~^2 + U~^2), Eq. pPhi).  Ties go to the lowest index;
 * NaN magnitudes are never selected; a row with no finite magnitude gives -1.
 *   F : [nlos][nphi][2];  idx : [nlos];  absF : [nlos] (NaN when idx == -1)
 */
void oracle_peak(int64_t nlos, int32_t nphi, const double *F, int32_t *idx, double *absF)
{
#pragma omp parallel for schedule(static)
    for (int64_t l = 0; l < nlos; ++l) {
        const double *Fl = F + (size_t)l * (size_t)nphi * 2;
        int32_t best = -1;
        double bestm = 0.0;
        for (int32_t k = 0; k < nphi; ++k) {
            double m = sqrt(Fl[2 * k] * Fl[2 * k] + Fl[2 * k + 1] * Fl[2 * k + 1]);
            if (isnan(m)) continue;
            if (best < 0 || m > bestm) { best = k; bestm = m; }
        }
        idx[l] = best;
        absF[l] = best < 0 ? NAN : bestm;
    }
}
