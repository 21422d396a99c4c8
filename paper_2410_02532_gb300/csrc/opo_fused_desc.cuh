// opo_fused_desc.cuh -- per-instance descriptor of the fused kernels and the
// kernel that turns their per-CTA observable sums into the trace.
#pragma once

#include "opo_common.cuh"
#include "opo_internal.h"

namespace opo {

struct InstDesc {
    void *fields;      // F*N state (read at start, written at end)
    void *out;         // F*N output-coupled fields of the last round trip
    void *hist;        // output history rows [slot][F*N], or null
    const void *pump;  // N input pump
    const void *disp;  // F*N dispersion factors / N (natural order)
    const void *gdd;   // F*N cavity spectral factors / N (natural order)
    const void *disp_t; // the same two tables row-major over N = P Q:
    const void *gdd_t;  //   [x][k1][k2] holds bin k1 + k2 P
    const void *tw;    // N twiddles W_N^j
    const void *ekz;   // 4 nz + 1 factors e^{i dk q dz/4}
    double *obs;       // raw sums of slot 0 of this call: [slot][C][kNslot]
    double *trace;     // rows {P_p, P_s, P_i, nu_c} of this call
    int *err;          // sticky error word
    int n, logn, logP, logQ, F, nz;
    unsigned resmask;
    int use_dk, eom;
    double kappa[3], h;
    double bc_re[3], bc_im[3], outscale[3];
    double eom_beta, eom_f, t_rt, dt, t_window;
    double pscale[3];  // n eps0 c / 2 * pi w0^2
    int64_t m_start;   // round-trip counter at the start of the call
    NsPump ns;         // ns-pulsed pump (ns.on), replaces the pump table
    int kerr;          // chi(3) terms on
    double kerr_g[9];  // their coefficients G_xy, row-major
    const CryDesc *cry; // every crystal of the round trip (cry[0]: the fields above)
    int ncry;
    void *xg1, *xg2;   // F*N each: exchange buffers of the form that exchanges
                       // through global memory (null where unused)
};

// Observables of every instance and slot of the call: output power
// (1/N) Sum|A|^2 (1 - R) n eps0 c/2 pi w0^2 and the signal centroid
// Sum k'|X_k|^2 / Sum |X_k|^2 / T, reduced over the C partial sums in a fixed
// order.
static __global__ void k_finalize_fused(const InstDesc *__restrict__ descs, int count, int C, int M)
{
    const int64_t total = (int64_t)count * M;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(t / M), s = (int)(t % M);
        const InstDesc &d = descs[i];
        double sum[kNslot] = {0, 0, 0, 0, 0};
        for (int c = 0; c < C; c++)
            for (int q = 0; q < kNslot; q++)
                sum[q] += d.obs[((int64_t)s * C + c) * kNslot + q];
        const double inv_n = 1.0 / (double)d.n;
        for (int x = 0; x < 3; x++)
            d.trace[(int64_t)s * 4 + x] =
                (x < d.F) ? sum[x] * inv_n * d.outscale[x] * d.outscale[x] * d.pscale[x] : 0.0;
        d.trace[(int64_t)s * 4 + 3] = sum[3] > 0.0 ? (sum[4] / sum[3]) / d.t_window : 0.0;
    }
}


// Sum five per-thread FP64 values over the block; thread 0 gets the totals.
static __device__ __forceinline__ void block_reduce5(double *v, double *red)
{
    for (int q = 0; q < kNslot; q++)
        for (int o = 16; o > 0; o >>= 1)
            v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0)
        for (int q = 0; q < kNslot; q++)
            red[w * kNslot + q] = v[q];
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int q = 0; q < kNslot; q++) {
            double t = 0.0;
            for (int i = 0; i < (int)(blockDim.x >> 5); i++)
                t += red[i * kNslot + q];
            v[q] = t;
        }
    }
}

// Fill one descriptor from a context (host).
void fill_desc(InstDesc &d, const opo_ctx *c);

// opo_fused2.cu: the size-specialised kernel (N = 2^12 .. 2^17, one size and
// field count per launch).
bool fused2_config(bool dbl, int nl, int F, int logn, int C, int threads_req, FusedCfg *out);
int fused2_max_active(bool dbl, int F, int logn, const FusedCfg &cfg);
int fused2_launch(bool dbl, int F, int logn, const InstDesc *dd, int count, const FusedCfg &cfg,
                  int r_base, int chunk, int last, cudaStream_t s);

} // namespace opo
