/*
 * opo_oracle.h -- plain FP64 CPU oracle of the OPO split-step hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load or call this code.  The
 * product library (libopo.so) neither includes this header nor links this
 * object; the two share no code, tables or constants.
 *
 * Method (arXiv 2410.02532):
 *   - coupled-wave equations, Sec. 2.1 Eqs. (CEp)-(CEi), linear operator
 *     Eq. (linearop);
 *   - symmetrized split-step N/2 - L - N/2 with RK4 for the nonlinear part,
 *     Sec. 2.2 Eq. (expon) and the field-evolution formula after it;
 *   - cavity boundary condition Eq. (BC), Sec. 2.1;
 *   - intracavity GDD and EOM, Sec. 2.3 items 1 and 2, applied in the order of
 *     the main-loop listing of Sec. 4.1 (GDD, then mirror, then EOM);
 *   - grid dt = t_rt/n, dnu = 1/t_rt, Sec. 2.4.
 *
 * Field index: 0 = pump, 1 = signal, 2 = idler.  Two-field mode (degenerate,
 * Sec. 4.4) uses 0 = pump and 1 = signal.
 *
 * Arrays at this interface are interleaved (re, im) doubles.
 */
#ifndef OPO_ORACLE_H
#define OPO_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Parameters of one nonlinear crystal of the round trip (the same meaning
 * as the crystal fields of orc_params). */
typedef struct {
    double  length;
    int32_t nz;
    double  dk;
    double  deff;
    double  nidx[3];
    double  alpha[3];
    double  dbeta1[3];
    double  beta2[3];
    double  beta3[3];
    double  beta4[3];
    double  tod_div;
    double  n2;
} orc_crystal;

#define ORC_MAX_EXTRA 7

typedef struct {
    int32_t n;              /* grid points N (power of two)                       */
    int32_t nfields;        /* 2 (degenerate) or 3                                */
    double  t_window;       /* window T = t_rt [s]; dt = T/N (Sec. 2.4)           */
    /* crystal */
    double  length;         /* L [m]                                              */
    int32_t nz;             /* fixed z-steps per pass (Sec. 2.4, 50..250)         */
    double  dk;             /* Delta k [1/m]                                      */
    double  deff;           /* d_eff [m/V]                                        */
    double  lambda[3];      /* vacuum wavelengths [m]                             */
    double  nidx[3];        /* refractive indices                                 */
    double  alpha[3];       /* power attenuation alpha_x [1/m]                    */
    double  dbeta1[3];      /* 1/nu_x - 1/nu_s [s/m]                              */
    double  beta2[3];       /* k''_x [s^2/m]                                      */
    double  beta3[3];       /* k'''_x [s^3/m]                                     */
    double  tod_div;        /* divisor of the beta3 term: 6 (Taylor)              */
    double  w0;             /* pump waist for power <-> intensity [m]             */
    /* cavity */
    uint32_t resonant_mask; /* bit x set: field x is resonant                     */
    double  R[3];           /* mirror power reflectivity 1 - theta_x              */
    double  delta[3];       /* detuning phase delta_x [rad]                       */
    double  gdd[3];         /* intracavity GDD gamma_x [s^2]                      */
    double  delay;          /* per-round-trip timing mismatch Delta t [s]         */
    double  eom_beta;       /* EOM depth beta [rad]                               */
    double  eom_f;          /* EOM frequency f_pm [Hz]                            */
    double  t_rt;           /* round-trip time for the EOM phase [s]              */
    /* ns-pulsed pump (Sec. 4.2): a Gaussian much longer than t_rt, sliced
     * per round trip; used instead of pump_in when ns_fwhm > 0 */
    double  ns_a0;          /* peak field amplitude [V/m]                         */
    double  ns_fwhm;        /* intensity FWHM [s]                                 */
    double  ns_t0;          /* pulse centre on the round-trip time axis [s]       */
    /* chi(3) and higher-order dispersion (named as extensions in Sec. 1 and
     * Sec. 2.1): fourth-order dispersion and the Kerr index */
    double  beta4[3];       /* fourth derivative of k_x [s^4/m]                   */
    double  n2;             /* Kerr index [m^2/W]; 0: no chi(3) terms             */
    /* further crystals passed after the first one in every round trip
     * (Sec. 5: one or more nonlinear media in the cavity); the fields go on
     * unchanged from one crystal to the next and z restarts at 0 in each */
    int32_t nextra;
    orc_crystal extra[ORC_MAX_EXTRA];
} orc_params;

/* In-place DFT of length n (power of two).  dir = -1: forward, unnormalized,
 * X_k = sum_n A_n exp(-2 pi i k n / N).  dir = +1: inverse, with 1/N.
 * Returns 0, or -1 if n is not a power of two. */
int orc_fft(double *z, int32_t n, int32_t dir);

/* kappa_x = 2 pi d_eff / (n_x lambda_x), Sec. 2.1 after Eq. (CEi). */
void orc_kappa(const orc_params *p, double kappa_out[3]);

/* Angular frequency offset of bin k in FFT order: 2 pi k'/T. */
double orc_omega(const orc_params *p, int32_t k);

/* Linear step over dz on every field: A <- F^-1[ D(Omega) F[A] ], with
 * D = exp{dz [-alpha/2 + i(-dbeta1 W + beta2 W^2/2 - beta3 W^3/tod_div
 *                          + beta4 W^4/24)]}. */
void orc_linear_step(const orc_params *p, double *fields, double dz);

/* One classic RK4 step of size h from z0 on the pointwise nonlinear system:
 * the chi(2) terms of Eqs. (CEp)-(CEi) plus, when n2 != 0, self- and
 * cross-phase modulation i k0_x n2 (I_x + 2 sum_{y != x} I_y) A_x with
 * I_y = n_y eps0 c |A_y|^2 / 2 and k0_x = 2 pi / lambda_x. */
void orc_rk4_step(const orc_params *p, double *fields, double z0, double h);

/* One crystal pass: nz symmetrized steps N/2 - L - N/2. */
void orc_crystal_pass(const orc_params *p, double *fields);

/* q <- p with the crystal fields replaced by those of crystal k (0: the
 * first crystal, i.e. p itself; 1..nextra: extra[k-1]). */
void orc_crystal_k(const orc_params *p, int32_t k, orc_params *q);

/* Input pump profile.  kind 0: CW, 1: sech^2 (peak power), power [W],
 * fwhm [s] (intensity FWHM, sech^2 only).  out: n complex values. */
void orc_pump_profile(const orc_params *p, int32_t kind, double power,
                      double fwhm, double *out);

/* Power carried by a field: mean |A|^2 * (1/2) n eps0 c * pi w0^2. */
double orc_power(const orc_params *p, int32_t field, const double *a);

/* Spectral centroid sum_k f_k |X_k|^2 / sum_k |X_k|^2 [Hz], f_k = k'/T. */
double orc_centroid(const orc_params *p, const double *a);

/* Apply the cavity elements of Sec. 2.3 / Eq. (BC) to resonant fields at
 * round trip m (GDD and delay, mirror, EOM). */
void orc_cavity(const orc_params *p, double *fields, int64_t m);

/* Input pump of round trip m (n complex): pump_in, or the slice
 * t = m t_rt + tau_n of the ns-pulsed pump when ns_fwhm > 0. */
void orc_pump_slice(const orc_params *p, const double *pump_in, int64_t m, double *out);

/* Run round trips m0 .. m0+M-1.  fields: F*n complex, in/out (state at the
 * start of the next round trip).  pump_in: n complex (ignored for an
 * ns-pulsed pump).  Entry: a non-resonant pump is replaced by the input
 * pump, a resonant pump (pump-resonant cavity) gets it added.  The crystal
 * pass goes through crystal 0, then the extra crystals in order.  trace (optional):
 * M rows of {P_p_out, P_s_out, P_i_out, nu_c}.  out_fields (optional): F*n
 * complex output-coupled fields of the last round trip.  Returns 0, or 1 if a
 * non-finite value appeared (the run stops at that round trip). */
int orc_run(const orc_params *p, double *fields, const double *pump_in,
            int64_t m0, int64_t M, double *trace, double *out_fields);

#ifdef __cplusplus
}
#endif
#endif
