/*
 * opo_oracle.c -- plain, slow, single-threaded FP64 oracle of the OPO
 * split-step Fourier hot path (arXiv 2410.02532).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load or call this code.  It
 * shares no code, header, table or constant with the CUDA library.
 *
 * Every step follows the paper's definitions in the paper's order, with no
 * blocking, fusion or reordering:
 *   grid .................... Sec. 2.4 (dt = t_rt/n, dnu = 1/t_rt)
 *   DFT ..................... textbook radix-2 decimation in time, own code
 *   linear operator ......... Sec. 2.1 Eq. (linearop), applied in the
 *                             frequency domain (Sec. 2.2)
 *   nonlinear operator ...... Sec. 2.1 Eqs. (CEp)-(CEi), RK4 (Sec. 2.2)
 *   split step .............. Sec. 2.2 Eq. (expon): N/2 - L - N/2
 *   boundary condition ...... Sec. 2.1 Eq. (BC)
 *   intracavity elements .... Sec. 2.3 items 1 (GDD) and 2 (EOM), in the
 *                             order of the main-loop listing of Sec. 4.1
 *
 * Readings where the paper is silent or garbled (each one is tested):
 *   - third-order dispersion uses the Taylor factor 1/6 (the printed 1/3 is
 *     kept reachable through tod_div);
 *   - group-velocity mismatch moves a field slower than the signal to later
 *     times; the Fourier convention is X_k = sum_n A_n e^{-2 pi i k n/N}, so
 *     d/dtau <-> +i Omega;
 *   - two-field (degenerate) pump equation dA_p/dz = i (kappa_p/2) A_s^2
 *     e^{-i dk z}, the factor 1/2 forced by power conservation;
 *   - non-resonant signal/idler restart from zero at every crystal entry;
 *   - z in e^{i dk z} is the position inside the crystal;
 *   - GDD is transformed back with the inverse transform;
 *   - the EOM phase uses tau_n = (n - N/2) dt plus m t_rt;
 *   - a resonant pump (pump-resonant cavity) gets the input pump added at
 *     entry; an ns-pulsed pump is a Gaussian in intensity read at
 *     t = m t_rt + tau_n.
 * Parity unpinned (no printed values survive): the paper's figure curves,
 * its ns-pulsed example and its absolute threshold powers.
 */
#include "opo_oracle.h"

#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_PI 3.141592653589793238462643383279502884
static const double EPS0 = 8.8541878128e-12; /* vacuum permittivity [F/m] */
static const double C0 = 299792458.0;        /* speed of light [m/s]      */

/* ---------------------------------------------------------------- DFT --- */

static int is_pow2(int32_t n) { return n > 0 && (n & (n - 1)) == 0; }

int orc_fft(double *z, int32_t n, int32_t dir)
{
    if (!is_pow2(n))
        return -1;
    double complex *a = (double complex *)z;
    /* bit-reversal permutation */
    for (int32_t i = 1, j = 0; i < n; i++) {
        int32_t bit = n >> 1;
        for (; j & bit; bit >>= 1)
            j ^= bit;
        j ^= bit;
        if (i < j) {
            double complex t = a[i];
            a[i] = a[j];
            a[j] = t;
        }
    }
    double complex *w = (double complex *)malloc(sizeof(double complex) * (size_t)(n / 2 + 1));
    /* butterflies of growing length; twiddles e^{dir 2 pi i k/len} */
    for (int32_t len = 2; len <= n; len <<= 1) {
        int32_t half = len / 2;
        for (int32_t k = 0; k < half; k++) {
            double ang = (double)dir * 2.0 * ORC_PI * (double)k / (double)len;
            w[k] = cos(ang) + I * sin(ang);
        }
        for (int32_t i = 0; i < n; i += len) {
            for (int32_t k = 0; k < half; k++) {
                double complex u = a[i + k];
                double complex v = a[i + k + half] * w[k];
                a[i + k] = u + v;
                a[i + k + half] = u - v;
            }
        }
    }
    free(w);
    if (dir > 0) {
        for (int32_t i = 0; i < n; i++)
            a[i] /= (double)n;
    }
    return 0;
}

/* --------------------------------------------------------------- grid --- */

double orc_omega(const orc_params *p, int32_t k)
{
    int32_t kk = (k < p->n / 2) ? k : k - p->n;
    return 2.0 * ORC_PI * (double)kk / p->t_window;
}

static double tau_of(const orc_params *p, int32_t idx)
{
    double dt = p->t_window / (double)p->n;
    return (double)(idx - p->n / 2) * dt;
}

void orc_kappa(const orc_params *p, double kappa_out[3])
{
    for (int x = 0; x < 3; x++)
        kappa_out[x] = (p->lambda[x] > 0.0 && p->nidx[x] > 0.0)
                           ? 2.0 * ORC_PI * p->deff / (p->nidx[x] * p->lambda[x])
                           : 0.0;
}

/* ----------------------------------------------------- linear operator --- */

/* D_x(Omega) = exp{ dz [ -alpha/2 + i(-dbeta1 Omega + beta2 Omega^2/2
 *                                     - beta3 Omega^3/tod_div
 *                                     + beta4 Omega^4/24) ] }
 * (Taylor series of the propagation constant: with d/dtau <-> +i Omega the
 * term of order k carries i (-1)^k beta_k Omega^k / k!)                   */
static double complex dispersion_factor(const orc_params *p, int x, double om, double dz)
{
    double phase = -p->dbeta1[x] * om + p->beta2[x] * om * om / 2.0
                   - p->beta3[x] * om * om * om / p->tod_div
                   + p->beta4[x] * om * om * om * om / 24.0;
    double amp = exp(-p->alpha[x] * dz / 2.0);
    return amp * (cos(phase * dz) + I * sin(phase * dz));
}

void orc_linear_step(const orc_params *p, double *fields, double dz)
{
    int32_t n = p->n;
    for (int x = 0; x < p->nfields; x++) {
        double *a = fields + (size_t)2 * n * x;
        orc_fft(a, n, -1);
        double complex *ac = (double complex *)a;
        for (int32_t k = 0; k < n; k++)
            ac[k] *= dispersion_factor(p, x, orc_omega(p, k), dz);
        orc_fft(a, n, +1);
    }
}

/* -------------------------------------------------- nonlinear operator --- */

/* Right-hand side of Eqs. (CEp)-(CEi) without the linear part at one point. */
static void nl_rhs(const orc_params *p, const double kap[3], const double complex *A,
                   double z, double complex *f)
{
    double complex e = cos(p->dk * z) + I * sin(p->dk * z); /* e^{+i dk z} */
    if (p->nfields == 3) {
        f[0] = I * kap[0] * A[1] * A[2] * conj(e);
        f[1] = I * kap[1] * A[0] * conj(A[2]) * e;
        f[2] = I * kap[2] * A[0] * conj(A[1]) * e;
    } else {
        f[0] = I * (kap[0] / 2.0) * A[1] * A[1] * conj(e);
        f[1] = I * kap[1] * A[0] * conj(A[1]) * e;
    }
    if (p->n2 != 0.0) {
        /* Kerr: intensity-dependent index n2 I; a co-propagating field at
         * another frequency counts twice (cross-phase modulation) */
        double inten[3];
        for (int x = 0; x < p->nfields; x++)
            inten[x] = 0.5 * p->nidx[x] * EPS0 * C0 * creal(A[x] * conj(A[x]));
        for (int x = 0; x < p->nfields; x++) {
            double itot = inten[x];
            for (int y = 0; y < p->nfields; y++)
                if (y != x)
                    itot += 2.0 * inten[y];
            double k0 = 2.0 * ORC_PI / p->lambda[x];
            f[x] += I * k0 * p->n2 * itot * A[x];
        }
    }
}

void orc_rk4_step(const orc_params *p, double *fields, double z0, double h)
{
    int32_t n = p->n;
    int F = p->nfields;
    double kap[3];
    orc_kappa(p, kap);
    double complex *A[3];
    for (int x = 0; x < F; x++)
        A[x] = (double complex *)(fields + (size_t)2 * n * x);
    for (int32_t j = 0; j < n; j++) {
        double complex y[3] = {0}, t[3] = {0}, k1[3], k2[3], k3[3], k4[3];
        for (int x = 0; x < F; x++)
            y[x] = A[x][j];
        nl_rhs(p, kap, y, z0, k1);
        for (int x = 0; x < F; x++)
            t[x] = y[x] + (h / 2.0) * k1[x];
        nl_rhs(p, kap, t, z0 + h / 2.0, k2);
        for (int x = 0; x < F; x++)
            t[x] = y[x] + (h / 2.0) * k2[x];
        nl_rhs(p, kap, t, z0 + h / 2.0, k3);
        for (int x = 0; x < F; x++)
            t[x] = y[x] + h * k3[x];
        nl_rhs(p, kap, t, z0 + h, k4);
        for (int x = 0; x < F; x++)
            A[x][j] = y[x] + (h / 6.0) * (k1[x] + 2.0 * k2[x] + 2.0 * k3[x] + k4[x]);
    }
}

/* ------------------------------------------------------- crystal pass --- */

void orc_crystal_pass(const orc_params *p, double *fields)
{
    double dz = p->length / (double)p->nz;
    for (int32_t j = 0; j < p->nz; j++) {
        double zj = (double)j * dz;
        orc_rk4_step(p, fields, zj, dz / 2.0);
        orc_linear_step(p, fields, dz);
        orc_rk4_step(p, fields, zj + dz / 2.0, dz / 2.0);
    }
}

void orc_crystal_k(const orc_params *p, int32_t k, orc_params *q)
{
    *q = *p;
    if (k < 1 || k > p->nextra)
        return;
    const orc_crystal *c = &p->extra[k - 1];
    q->length = c->length;
    q->nz = c->nz;
    q->dk = c->dk;
    q->deff = c->deff;
    for (int x = 0; x < 3; x++) {
        q->nidx[x] = c->nidx[x];
        q->alpha[x] = c->alpha[x];
        q->dbeta1[x] = c->dbeta1[x];
        q->beta2[x] = c->beta2[x];
        q->beta3[x] = c->beta3[x];
        q->beta4[x] = c->beta4[x];
    }
    q->tod_div = c->tod_div;
    q->n2 = c->n2;
}

/* ---------------------------------------------------------- pump / obs --- */

void orc_pump_profile(const orc_params *p, int32_t kind, double power, double fwhm, double *out)
{
    double intensity = power / (ORC_PI * p->w0 * p->w0);
    double a0 = sqrt(2.0 * intensity / (p->nidx[0] * EPS0 * C0));
    double t0 = fwhm / (2.0 * acosh(sqrt(2.0))); /* sech^2 intensity FWHM */
    for (int32_t j = 0; j < p->n; j++) {
        double amp = a0;
        if (kind == 1)
            amp = a0 / cosh(tau_of(p, j) / t0);
        out[2 * j] = amp;
        out[2 * j + 1] = 0.0;
    }
}

double orc_power(const orc_params *p, int32_t field, const double *a)
{
    double s = 0.0;
    for (int32_t j = 0; j < p->n; j++)
        s += a[2 * j] * a[2 * j] + a[2 * j + 1] * a[2 * j + 1];
    double mean = s / (double)p->n;
    return mean * 0.5 * p->nidx[field] * EPS0 * C0 * ORC_PI * p->w0 * p->w0;
}

double orc_centroid(const orc_params *p, const double *a)
{
    int32_t n = p->n;
    double *x = (double *)malloc(sizeof(double) * 2 * (size_t)n);
    memcpy(x, a, sizeof(double) * 2 * (size_t)n);
    orc_fft(x, n, -1);
    double num = 0.0, den = 0.0;
    for (int32_t k = 0; k < n; k++) {
        int32_t kk = (k < n / 2) ? k : k - n;
        double pk = x[2 * k] * x[2 * k] + x[2 * k + 1] * x[2 * k + 1];
        num += ((double)kk / p->t_window) * pk;
        den += pk;
    }
    free(x);
    return den > 0.0 ? num / den : 0.0;
}

/* ------------------------------------------------------------- cavity --- */

void orc_cavity(const orc_params *p, double *fields, int64_t m)
{
    int32_t n = p->n;
    for (int x = 0; x < p->nfields; x++) {
        if (!(p->resonant_mask & (1u << x)))
            continue;
        double complex *a = (double complex *)(fields + (size_t)2 * n * x);
        /* Sec. 2.3 item 1: GDD e^{i gamma Omega^2/2}, and the timing mismatch
         * e^{-i Omega dt}, in the frequency domain */
        if (p->gdd[x] != 0.0 || p->delay != 0.0) {
            orc_fft((double *)a, n, -1);
            for (int32_t k = 0; k < n; k++) {
                double om = orc_omega(p, k);
                double ph = p->gdd[x] * om * om / 2.0 - om * p->delay;
                a[k] *= cos(ph) + I * sin(ph);
            }
            orc_fft((double *)a, n, +1);
        }
        /* Eq. (BC): sqrt(1 - theta) e^{i delta} */
        double complex bc = sqrt(p->R[x]) * (cos(p->delta[x]) + I * sin(p->delta[x]));
        for (int32_t j = 0; j < n; j++)
            a[j] *= bc;
        /* Sec. 2.3 item 2: EOM e^{i beta sin(2 pi f_pm tau)}, tau = tau_n + m t_rt */
        if (p->eom_beta != 0.0) {
            for (int32_t j = 0; j < n; j++) {
                double u = p->eom_f * (tau_of(p, j) + (double)m * p->t_rt);
                double fr = u - floor(u);
                double ph = p->eom_beta * sin(2.0 * ORC_PI * fr);
                a[j] *= cos(ph) + I * sin(ph);
            }
        }
    }
}

/* ---------------------------------------------------- ns-pulsed pump --- */

/* Gaussian in intensity with FWHM ns_fwhm: A(t) = a0 exp(-2 ln 2 (t - t0)^2
 * / fwhm^2), sampled at t = m t_rt + tau_n (Sec. 4.2: the long input pump
 * is read one round trip at a time). */
void orc_pump_slice(const orc_params *p, const double *pump_in, int64_t m, double *out)
{
    if (!(p->ns_fwhm > 0.0)) {
        memcpy(out, pump_in, sizeof(double) * 2 * (size_t)p->n);
        return;
    }
    for (int32_t j = 0; j < p->n; j++) {
        double t = (double)m * p->t_rt + tau_of(p, j) - p->ns_t0;
        out[2 * j] = p->ns_a0 * exp(-2.0 * log(2.0) * t * t / (p->ns_fwhm * p->ns_fwhm));
        out[2 * j + 1] = 0.0;
    }
}

/* ---------------------------------------------------------- round trip --- */

static int all_finite(const double *v, size_t cnt)
{
    for (size_t i = 0; i < cnt; i++)
        if (!isfinite(v[i]))
            return 0;
    return 1;
}

int orc_run(const orc_params *p, double *fields, const double *pump_in,
            int64_t m0, int64_t M, double *trace, double *out_fields)
{
    int32_t n = p->n;
    int F = p->nfields;
    size_t fsz = (size_t)2 * n;
    double *outbuf = (double *)malloc(sizeof(double) * fsz);
    double *pump = (double *)malloc(sizeof(double) * fsz);
    for (int64_t r = 0; r < M; r++) {
        int64_t m = m0 + r;
        /* entry: the input pump replaces a non-resonant pump and is added to a
         * resonant one; non-resonant signal/idler restart from 0 */
        orc_pump_slice(p, pump_in, m, pump);
        for (int x = 0; x < F; x++) {
            double *a = fields + fsz * x;
            if (p->resonant_mask & (1u << x)) {
                if (x == 0)
                    for (size_t i = 0; i < fsz; i++)
                        a[i] += pump[i];
                continue;
            }
            if (x == 0)
                memcpy(a, pump, sizeof(double) * fsz);
            else
                memset(a, 0, sizeof(double) * fsz);
        }
        for (int32_t k = 0; k <= p->nextra; k++) {
            orc_params q;
            orc_crystal_k(p, k, &q);
            orc_crystal_pass(&q, fields);
        }
        /* output-coupled fields and per-round-trip observables */
        double rec[4] = {0.0, 0.0, 0.0, 0.0};
        for (int x = 0; x < F; x++) {
            double *a = fields + fsz * x;
            double s = (p->resonant_mask & (1u << x)) ? sqrt(1.0 - p->R[x]) : 1.0;
            for (size_t i = 0; i < fsz; i++)
                outbuf[i] = s * a[i];
            rec[x] = orc_power(p, x, outbuf);
            if (x == 1)
                rec[3] = orc_centroid(p, outbuf);
            if (out_fields != NULL && r == M - 1)
                memcpy(out_fields + fsz * x, outbuf, sizeof(double) * fsz);
        }
        if (trace != NULL)
            memcpy(trace + 4 * r, rec, sizeof(rec));
        if (!all_finite(fields, fsz * (size_t)F)) {
            free(outbuf);
            free(pump);
            return 1;
        }
        orc_cavity(p, fields, m);
    }
    free(outbuf);
    free(pump);
    return 0;
}
