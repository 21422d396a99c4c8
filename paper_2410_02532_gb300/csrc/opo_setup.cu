// opo_setup.cu -- per-instance tables built on the device from FP64
// arguments and rounded once to the field precision:
//   twiddles W_N^j = e^{-2 pi i j/N};
//   dispersion factor of one z-step, Eq. (linearop) of arXiv 2410.02532 in
//     the frequency domain (Sec. 2.2), with the inverse-FFT 1/N folded in;
//   cavity spectral factor: GDD e^{i gamma Omega^2/2} (Sec. 2.3 item 1) and
//     the timing mismatch e^{-i Omega delay}, with 1/N folded in;
//   e^{i dk z} at the RK4 stage positions z = q dz/4 (Eqs. (CEp)-(CEi));
//   the input pump (CW, sech^2 or user profile);
// and the per-round-trip observables (power, signal spectral centroid).
#include "opo_common.cuh"
#include "opo_internal.h"

namespace opo {
namespace {

template <class T>
__global__ void k_twiddles(cv<T> *tw, int n)
{
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        double s, c;
        sincospi(-2.0 * (double)j / (double)n, &s, &c);
        tw[j] = cmk<cv<T>>((T)c, (T)s);
    }
}

struct DispArgs {
    double alpha[3], db1[3], b2[3], b3[3], b4[3];
    double tod_div, dz, t_window;
};

__device__ __forceinline__ double omega_k(int k, int n, double t_window)
{
    int kk = (k < n / 2) ? k : k - n;
    return 2.0 * kPi * (double)kk / t_window;
}

// Index of bin k of field x in the row-major copy: [x][k1][k2], k = k1 + k2 P.
__device__ __forceinline__ int rowmajor_index(int x, int k, int n, int logP)
{
    const int logQ = ilog2((unsigned)n) - logP;
    return x * n + ((k & ((1 << logP) - 1)) << logQ) + (k >> logP);
}

// Dt (optional): the row-major copy, over N = 2^logP x N/2^logP.
template <class T>
__global__ void k_disp_table(cv<T> *D, cv<T> *Dt, int logP, int n, int F, DispArgs a)
{
    const double inv_n = 1.0 / (double)n;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < F * n; i += gridDim.x * blockDim.x) {
        int x = i / n, k = i % n;
        double om = omega_k(k, n, a.t_window);
        double ph = a.dz * (-a.db1[x] * om + a.b2[x] * om * om * 0.5
                            - a.b3[x] * om * om * om / a.tod_div
                            + a.b4[x] * om * om * om * om / 24.0);
        double amp = exp(-a.alpha[x] * a.dz * 0.5) * inv_n;
        double s, c;
        sincos(ph, &s, &c);
        const cv<T> d = cmk<cv<T>>((T)(amp * c), (T)(amp * s));
        D[i] = d;
        if (Dt)
            Dt[rowmajor_index(x, k, n, logP)] = d;
    }
}

struct GddArgs {
    double gdd[3];
    double delay, t_window;
    unsigned resmask;
};

template <class T>
__global__ void k_gdd_table(cv<T> *G, cv<T> *Gt, int logP, int n, int F, GddArgs a)
{
    const double inv_n = 1.0 / (double)n;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < F * n; i += gridDim.x * blockDim.x) {
        int x = i / n, k = i % n;
        double ph = 0.0;
        if (a.resmask & (1u << x)) {
            double om = omega_k(k, n, a.t_window);
            ph = a.gdd[x] * om * om * 0.5 - om * a.delay;
        }
        double s, c;
        sincos(ph, &s, &c);
        const cv<T> g = cmk<cv<T>>((T)(c * inv_n), (T)(s * inv_n));
        G[i] = g;
        Gt[rowmajor_index(x, k, n, logP)] = g;
    }
}

template <class T>
__global__ void k_ekz_table(cv<T> *E, int cnt, double dk, double dz)
{
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < cnt; q += gridDim.x * blockDim.x) {
        double s, c;
        sincos(dk * ((double)q * dz * 0.25), &s, &c);
        E[q] = cmk<cv<T>>((T)c, (T)s);
    }
}

template <class T>
__global__ void k_pump(cv<T> *p, int n, int kind, double a0, double t0, double dt,
                       const double *user)
{
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        double re = a0, im = 0.0;
        if (kind == OPO_PUMP_SECH2) {
            double tau = (double)(j - n / 2) * dt;
            re = a0 / cosh(tau / t0);
        } else if (kind == OPO_PUMP_USER) {
            re = user[2 * j];
            im = user[2 * j + 1];
        }
        p[j] = cmk<cv<T>>((T)re, (T)im);
    }
}

struct FinArgs {
    double outscale2[3], pscale[3];
    double inv_n, t_window;
    int parts, F;
};

__global__ void k_finalize(const double *obs, double *trace, int64_t M, FinArgs a)
{
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < M;
         s += (int64_t)gridDim.x * blockDim.x) {
        double sum[kNslot] = {0, 0, 0, 0, 0};
        for (int c = 0; c < a.parts; c++)
            for (int q = 0; q < kNslot; q++)
                sum[q] += obs[(s * a.parts + c) * kNslot + q];
        for (int x = 0; x < 3; x++)
            trace[s * 4 + x] = (x < a.F) ? sum[x] * a.inv_n * a.outscale2[x] * a.pscale[x] : 0.0;
        trace[s * 4 + 3] = sum[3] > 0.0 ? (sum[4] / sum[3]) / a.t_window : 0.0;
    }
}

int grid_for(int64_t work)
{
    int64_t b = (work + 255) / 256;
    return (int)(b < 1 ? 1 : (b > 4096 ? 4096 : b));
}

} // namespace

int setup_twiddles(opo_ctx *c)
{
    if (c->prec == OPO_FP64)
        k_twiddles<double><<<grid_for(c->n), 256, 0, c->stream>>>((double2 *)c->d_tw, c->n);
    else
        k_twiddles<float><<<grid_for(c->n), 256, 0, c->stream>>>((float2 *)c->d_tw, c->n);
    return cudaGetLastError() == cudaSuccess ? OPO_OK : OPO_E_CUDA;
}

// Kerr: dA_x/dz += i (sum_y G_xy |A_y|^2) A_x with
// G_xy = (2 pi / lambda_x) n2 (n_y eps0 c / 2) (1 if y = x, else 2).
bool kerr_coefficients(const opo_crystal &k, int F, double g[9])
{
    const bool on = k.n2_m2_per_W != 0.0;
    for (int x = 0; x < 3; x++)
        for (int y = 0; y < 3; y++)
            g[3 * x + y] = (on && x < F && y < F)
                               ? (2.0 * kPi / k.lambda_m[x]) * k.n2_m2_per_W *
                                     (0.5 * k.n[y] * kEps0 * kC0) * (x == y ? 1.0 : 2.0)
                               : 0.0;
    return on;
}

namespace {

int crystal_tables(opo_ctx *c, const opo_crystal &k, void *disp, void *disp_t, void *ekz)
{
    DispArgs a;
    for (int x = 0; x < 3; x++) {
        a.alpha[x] = k.alpha_per_m[x];
        a.db1[x] = k.dbeta1_s_per_m[x];
        a.b2[x] = k.beta2_s2_per_m[x];
        a.b3[x] = k.beta3_s3_per_m[x];
        a.b4[x] = k.beta4_s4_per_m[x];
    }
    a.tod_div = k.tod_div > 0.0 ? k.tod_div : 6.0;
    a.dz = k.length_m / (double)k.nz;
    a.t_window = c->grid.t_window_s;
    int cnt = 4 * k.nz + 1;
    if (c->prec == OPO_FP64) {
        k_disp_table<double><<<grid_for((int64_t)c->F * c->n), 256, 0, c->stream>>>(
            (double2 *)disp, (double2 *)disp_t, c->logn / 2, c->n, c->F, a);
        k_ekz_table<double><<<grid_for(cnt), 256, 0, c->stream>>>((double2 *)ekz, cnt,
                                                                   k.dk_per_m, a.dz);
    } else {
        k_disp_table<float><<<grid_for((int64_t)c->F * c->n), 256, 0, c->stream>>>(
            (float2 *)disp, (float2 *)disp_t, c->logn / 2, c->n, c->F, a);
        k_ekz_table<float><<<grid_for(cnt), 256, 0, c->stream>>>((float2 *)ekz, cnt,
                                                                  k.dk_per_m, a.dz);
    }
    return cudaGetLastError() == cudaSuccess ? OPO_OK : OPO_E_CUDA;
}

} // namespace

int setup_crystal_tables(opo_ctx *c)
{
    for (int i = 0; i < c->ncry; i++) {
        void *disp = i == 0 ? c->d_disp : c->xs[i].disp;
        void *disp_t = i == 0 ? c->d_disp_t : c->xs[i].disp_t;
        void *ekz = i == 0 ? c->d_ekz : c->xs[i].ekz;
        int rc = crystal_tables(c, c->cry[i], disp, disp_t, ekz);
        if (rc != OPO_OK)
            return rc;
        c->h_cry[i].disp = disp;
        c->h_cry[i].disp_t = disp_t;
        c->h_cry[i].ekz = ekz;
    }
    // the pageable source is staged before cudaMemcpyAsync returns
    if (cudaMemcpyAsync(c->d_cry, c->h_cry, sizeof(CryDesc) * c->ncry, cudaMemcpyHostToDevice,
                        c->stream) != cudaSuccess)
        return OPO_E_CUDA;
    return OPO_OK;
}

int setup_cavity_tables(opo_ctx *c)
{
    const opo_cavity &v = c->cavity;
    GddArgs g;
    for (int x = 0; x < 3; x++)
        g.gdd[x] = v.gdd_s2[x];
    g.delay = v.delay_s;
    g.t_window = c->grid.t_window_s;
    g.resmask = v.resonant_mask;
    double intensity = v.pump_power_W / (kPi * c->crystal.w0_m * c->crystal.w0_m);
    double a0 = sqrt(2.0 * intensity / (c->crystal.n[0] * kEps0 * kC0));
    double t0 = v.pump_fwhm_s > 0.0 ? v.pump_fwhm_s / (2.0 * acosh(sqrt(2.0))) : 1.0;
    double dt = c->grid.t_window_s / (double)c->n;
    if (c->prec == OPO_FP64) {
        k_gdd_table<double><<<grid_for((int64_t)c->F * c->n), 256, 0, c->stream>>>(
            (double2 *)c->d_gdd, (double2 *)c->d_gdd_t, c->logn / 2, c->n, c->F, g);
        k_pump<double><<<grid_for(c->n), 256, 0, c->stream>>>((double2 *)c->d_pump, c->n,
                                                                v.pump_kind, a0, t0, dt,
                                                                c->d_pump_user);
    } else {
        k_gdd_table<float><<<grid_for((int64_t)c->F * c->n), 256, 0, c->stream>>>(
            (float2 *)c->d_gdd, (float2 *)c->d_gdd_t, c->logn / 2, c->n, c->F, g);
        k_pump<float><<<grid_for(c->n), 256, 0, c->stream>>>((float2 *)c->d_pump, c->n,
                                                               v.pump_kind, a0, t0, dt,
                                                               c->d_pump_user);
    }
    return cudaGetLastError() == cudaSuccess ? OPO_OK : OPO_E_CUDA;
}

int setup_pass_tables(void *tw, void *disp, void *ekz, int n, int F, bool dbl,
                      const opo_crystal &k, double t_window, cudaStream_t s)
{
    DispArgs a;
    for (int x = 0; x < 3; x++) {
        a.alpha[x] = k.alpha_per_m[x];
        a.db1[x] = k.dbeta1_s_per_m[x];
        a.b2[x] = k.beta2_s2_per_m[x];
        a.b3[x] = k.beta3_s3_per_m[x];
        a.b4[x] = k.beta4_s4_per_m[x];
    }
    a.tod_div = k.tod_div > 0.0 ? k.tod_div : 6.0;
    a.dz = k.length_m / (double)k.nz;
    a.t_window = t_window;
    const int cnt = 4 * k.nz + 1;
    if (dbl) {
        k_twiddles<double><<<grid_for(n), 256, 0, s>>>((double2 *)tw, n);
        k_disp_table<double><<<grid_for((int64_t)F * n), 256, 0, s>>>((double2 *)disp, nullptr, 0, n, F, a);
        k_ekz_table<double><<<grid_for(cnt), 256, 0, s>>>((double2 *)ekz, cnt, k.dk_per_m, a.dz);
    } else {
        k_twiddles<float><<<grid_for(n), 256, 0, s>>>((float2 *)tw, n);
        k_disp_table<float><<<grid_for((int64_t)F * n), 256, 0, s>>>((float2 *)disp, nullptr, 0, n, F, a);
        k_ekz_table<float><<<grid_for(cnt), 256, 0, s>>>((float2 *)ekz, cnt, k.dk_per_m, a.dz);
    }
    return cudaGetLastError() == cudaSuccess ? OPO_OK : OPO_E_CUDA;
}

int finalize_trace(opo_ctx *c, int64_t M, int parts)
{
    if (M <= 0)
        return OPO_OK;
    FinArgs a;
    for (int x = 0; x < 3; x++) {
        a.outscale2[x] = c->dv.outscale[x] * c->dv.outscale[x];
        a.pscale[x] = c->dv.pscale[x];
    }
    a.inv_n = 1.0 / (double)c->n;
    a.t_window = c->grid.t_window_s;
    a.parts = parts;
    a.F = c->F;
    k_finalize<<<grid_for(M), 256, 0, c->stream>>>(c->d_obs, c->d_trace, M, a);
    return cudaGetLastError() == cudaSuccess ? OPO_OK : OPO_E_CUDA;
}

} // namespace opo
