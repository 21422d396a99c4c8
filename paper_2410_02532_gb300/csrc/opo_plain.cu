// opo_plain.cu -- the plain GPU form of one OPO round trip: one kernel per
// operation per z-step (arXiv 2410.02532, Sec. 2.2 and the main loop of
// Sec. 4.1), with fields in HBM/L2 between kernels.  A round trip is
//   entry | nz x [RK4(dz/2), FFT, D, IFFT, RK4(dz/2)] | power sums |
//   output copy | FFT, signal spectrum sums, cavity spectral factor, IFFT |
//   mirror + EOM | round-trip counter
// and is captured once into a CUDA graph that every round trip replays.
//
// The FFT of length N = P Q runs as two kernels (four-step decomposition,
// n = Q n1 + n2, k = k1 + P k2): P-point column transforms with the twiddle
// W_N^{n2 k1} written to scratch, then Q-point row transforms written back in
// natural order.  Each kernel transforms a batch of columns or rows in shared
// memory with Stockham stages of radix 2..16.
#include "opo_common.cuh"
#include "opo_internal.h"

namespace opo {
namespace {

constexpr int kThreads = 256;

// Round-trip entry: the input pump (table, or the ns-pulsed pump read at
// this round trip) replaces a non-resonant pump and is added to a resonant
// one; non-resonant signal/idler restart from zero.
template <class T>
__global__ void k_entry(cv<T> *fields, const cv<T> *pump, int n, int F, unsigned resmask,
                        NsPump ns, const DevCtl *ctl)
{
    const int64_t m = ctl->rt0 + ctl->slot;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < F * n; i += gridDim.x * blockDim.x) {
        const int x = i / n;
        const bool res = (resmask >> x) & 1u;
        if (x == 0) {
            const cv<T> pin = ns.on ? ns_pump_at<T>(ns, i, m) : pump[i];
            fields[i] = res ? cadd(fields[i], pin) : pin;
        } else if (!res) {
            fields[i] = cmk<cv<T>>((T)0, (T)0);
        }
    }
}

// Kerr coefficients G_xy (row-major) in the field precision.
template <class T> struct KerrG {
    T g[9];
};

template <class T>
KerrG<T> kerr_g(const double *g)
{
    KerrG<T> k;
    for (int i = 0; i < 9; i++)
        k.g[i] = (T)g[i];
    return k;
}

template <class T, int F>
__global__ void k_rk4(cv<T> *fields, int n, const cv<T> *ekz, int q0, T h, T k0, T k1, T k2,
                      bool use_e, bool kerr, KerrG<T> G)
{
    using V = cv<T>;
    const T kap[3] = {k0, k1, k2};
    V e0 = ekz[q0], e1 = ekz[q0 + 1], e2 = ekz[q0 + 2];
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        V y[F];
#pragma unroll
        for (int x = 0; x < F; x++)
            y[x] = fields[(size_t)x * n + j];
        if (kerr)
            rk4_point_kerr<F>(y, e0, e1, e2, kap, h, use_e, G.g);
        else
            rk4_point<F>(y, e0, e1, e2, kap, h, use_e);
#pragma unroll
        for (int x = 0; x < F; x++)
            fields[(size_t)x * n + j] = y[x];
    }
}

// Column pass: grid (Q/B, fields).  Loads columns n2 in [g B, g B + B) of
// x[Q n1 + n2], transforms over n1, multiplies W_N^{DIR n2 k1} and writes
// y[k1 Q + n2].
template <class T, int DIR>
__global__ void k_fft_cols(const cv<T> *__restrict__ in, cv<T> *__restrict__ out, int n, int P,
                           int Q, int logP, int logn, int B, const cv<T> *__restrict__ tw)
{
    using V = cv<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V *s0 = reinterpret_cast<V *>(smem_raw);
    V *s1 = s0 + B * P;
    const V *src = in + (size_t)blockIdx.y * n;
    V *dst = out + (size_t)blockIdx.y * n;
    const int n2b = blockIdx.x * B;
    for (int i = threadIdx.x; i < B * P; i += blockDim.x) {
        int b = i % B, n1 = i / B;
        s0[n1 * B + b] = src[(size_t)n1 * Q + n2b + b];
    }
    __syncthreads();
    RadixPlan pl = make_plan(logP);
    V *a = s0, *o = s1;
    int Ns = 1;
    auto addr = [B](int seq, int e) { return e * B + seq; };
    for (int s = 0; s < pl.nst; s++) {
        int lr = pl.lr[s];
        V *ob = o;
        auto st = [ob, B](int seq, int e, V v) { ob[e * B + seq] = v; };
        stockham_stage_lr<DIR, true>(lr, a, B, P, Ns, addr, st, tw, logn - (ilog2(Ns) + lr));
        __syncthreads();
        V *t = a;
        a = o;
        o = t;
        Ns <<= lr;
    }
    for (int i = threadIdx.x; i < B * P; i += blockDim.x) {
        int b = i % B, k1 = i / B;
        int n2 = n2b + b;
        V w = tw[((size_t)n2 * k1) & (n - 1)];
        if (DIR > 0)
            w.y = -w.y;
        dst[(size_t)k1 * Q + n2] = cmul(a[k1 * B + b], w);
    }
}

// Row pass: grid (P/B, fields).  Loads rows k1 in [h B, h B + B) of
// y[k1 Q + n2], transforms over n2 and writes X[k1 + P k2].
template <class T, int DIR>
__global__ void k_fft_rows(const cv<T> *__restrict__ in, cv<T> *__restrict__ out, int n, int P,
                           int Q, int logQ, int logn, int B, const cv<T> *__restrict__ tw)
{
    using V = cv<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int Lp = Q + 1; // padded row stride
    V *s0 = reinterpret_cast<V *>(smem_raw);
    V *s1 = s0 + B * Lp;
    const V *src = in + (size_t)blockIdx.y * n;
    V *dst = out + (size_t)blockIdx.y * n;
    const int k1b = blockIdx.x * B;
    for (int i = threadIdx.x; i < B * Q; i += blockDim.x) {
        int b = i / Q, n2 = i % Q;
        s0[b * Lp + n2] = src[(size_t)(k1b + b) * Q + n2];
    }
    __syncthreads();
    RadixPlan pl = make_plan(logQ);
    V *a = s0, *o = s1;
    int Ns = 1;
    auto addr = [Lp](int seq, int e) { return seq * Lp + e; };
    for (int s = 0; s < pl.nst; s++) {
        int lr = pl.lr[s];
        V *ob = o;
        auto st = [ob, Lp](int seq, int e, V v) { ob[seq * Lp + e] = v; };
        stockham_stage_lr<DIR, false>(lr, a, B, Q, Ns, addr, st, tw, logn - (ilog2(Ns) + lr));
        __syncthreads();
        V *t = a;
        a = o;
        o = t;
        Ns <<= lr;
    }
    for (int i = threadIdx.x; i < B * Q; i += blockDim.x) {
        int b = i % B, k2 = i / B;
        dst[(size_t)(k1b + b) + (size_t)P * k2] = a[b * Lp + k2];
    }
}

template <class T>
__global__ void k_mul_table(cv<T> *a, const cv<T> *__restrict__ tab, int total)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x)
        a[i] = cmul(a[i], tab[i]);
}

__device__ __forceinline__ double block_sum(double v, double *red)
{
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0)
        red[w] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0) {
        for (int i = 0; i < (int)(blockDim.x >> 5); i++)
            t += red[i];
    }
    return t;
}

// One block per field: Sum |A_x|^2 of the post-crystal field into the raw
// observable slot of this round trip; a non-finite sum sets the error word.
template <class T>
__global__ void k_power_sums(const cv<T> *fields, int n, DevCtl *ctl)
{
    __shared__ double red[32];
    const int x = blockIdx.x;
    double s = 0.0;
    for (int j = threadIdx.x; j < n; j += blockDim.x)
        s += (double)cabs2(fields[(size_t)x * n + j]);
    s = block_sum(s, red);
    if (threadIdx.x == 0) {
        ctl->obs[ctl->slot * kNslot + x] = s;
        if (!isfinite(s))
            atomicOr(&ctl->err, 1);
    }
}

// Signal spectrum in natural order: Sum |X_k|^2 and Sum k'|X_k|^2.
template <class T>
__global__ void k_spec_sums(const cv<T> *spec, int n, DevCtl *ctl)
{
    __shared__ double red[32];
    double s0 = 0.0, s1 = 0.0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        double p = (double)cabs2(spec[k]);
        int kk = (k < n / 2) ? k : k - n;
        s0 += p;
        s1 += (double)kk * p;
    }
    s0 = block_sum(s0, red);
    s1 = block_sum(s1, red);
    if (threadIdx.x == 0) {
        ctl->obs[ctl->slot * kNslot + 3] = s0;
        ctl->obs[ctl->slot * kNslot + 4] = s1;
    }
}

template <class T>
__global__ void k_save_output(const cv<T> *fields, cv<T> *out, int n, int F, T s0, T s1, T s2,
                              cv<T> *hist, const DevCtl *ctl)
{
    const T sc[3] = {s0, s1, s2};
    cv<T> *row = hist ? hist + (size_t)ctl->slot * F * n : nullptr; // history row of this round trip
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < F * n; i += gridDim.x * blockDim.x) {
        const cv<T> o = cscale(fields[i], sc[i / n]);
        out[i] = o;
        if (row)
            row[i] = o;
    }
}

struct CavArgs {
    double bc_re[3], bc_im[3];
    double eom_beta, eom_f, t_rt, dt;
    unsigned resmask;
    int eom;
};

// Mirror sqrt(R) e^{i delta} (Eq. (BC)) then the EOM phase (Sec. 2.3 item 2)
// on resonant fields; the EOM argument frac(f_pm (tau_n + m t_rt)) is formed
// in FP64.
template <class T>
__global__ void k_cavity_time(cv<T> *fields, int n, int F, CavArgs a, const DevCtl *ctl)
{
    using V = cv<T>;
    const int64_t m = ctl->rt0 + ctl->slot;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        V mod = cmk<V>((T)1, (T)0);
        if (a.eom) {
            double u = a.eom_f * ((double)(j - n / 2) * a.dt) + a.eom_f * ((double)m * a.t_rt);
            double fr = u - floor(u);
            T ph;
            if constexpr (sizeof(T) == 8)
                ph = (T)(a.eom_beta * sinpi(2.0 * fr));
            else
                ph = (T)a.eom_beta * sinpif((T)2 * (T)fr);
            T sn, cs;
            sincos(ph, &sn, &cs);
            mod = cmk<V>(cs, sn);
        }
        for (int x = 0; x < F; x++) {
            if (!(a.resmask & (1u << x)))
                continue;
            V v = fields[(size_t)x * n + j];
            v = cmul(v, cmk<V>((T)a.bc_re[x], (T)a.bc_im[x]));
            if (a.eom)
                v = cmul(v, mod);
            fields[(size_t)x * n + j] = v;
        }
    }
}

__global__ void k_end_rt(DevCtl *ctl)
{
    ctl->slot += 1;
}

int blocks_for(int64_t work)
{
    int64_t b = (work + kThreads - 1) / kThreads;
    return (int)(b < 1 ? 1 : (b > 1184 ? 1184 : b));
}

template <class T>
struct PlainFFT {
    int n, logn, P, Q, logP, logQ, Bc, Br;
    size_t smc, smr;
    const cv<T> *tw;
    void init(const opo_ctx *c)
    {
        n = c->n;
        logn = c->logn;
        logP = logn / 2;
        logQ = logn - logP;
        P = 1 << logP;
        Q = 1 << logQ;
        int seg = (sizeof(T) == 8) ? 4 : 8; // 64-byte column segments
        Bc = Q < seg ? Q : seg;
        Br = P < seg ? P : seg;
        smc = (size_t)2 * Bc * P * sizeof(cv<T>);
        smr = (size_t)2 * Br * (Q + 1) * sizeof(cv<T>);
        tw = (const cv<T> *)c->d_tw;
    }
    // the same plan for caller-given sizes and twiddle table
    void init_raw(int n_, int logn_, const cv<T> *tw_)
    {
        n = n_;
        logn = logn_;
        logP = logn / 2;
        logQ = logn - logP;
        P = 1 << logP;
        Q = 1 << logQ;
        int seg = (sizeof(T) == 8) ? 4 : 8;
        Bc = Q < seg ? Q : seg;
        Br = P < seg ? P : seg;
        smc = (size_t)2 * Bc * P * sizeof(cv<T>);
        smr = (size_t)2 * Br * (Q + 1) * sizeof(cv<T>);
        tw = tw_;
    }
    // transform `count` consecutive fields of `a` in place, scratch `s`
    template <int DIR>
    void run(cv<T> *a, cv<T> *s, int count, cudaStream_t st) const
    {
        dim3 gc(Q / Bc, count), gr(P / Br, count);
        k_fft_cols<T, DIR><<<gc, kThreads, smc, st>>>(a, s, n, P, Q, logP, logn, Bc, tw);
        k_fft_rows<T, DIR><<<gr, kThreads, smr, st>>>(s, a, n, P, Q, logQ, logn, Br, tw);
    }
};

template <class T>
int enqueue_rt(opo_ctx *c, cudaStream_t st)
{
    using V = cv<T>;
    const int n = c->n, F = c->F;
    V *fld = (V *)c->d_fields;
    V *scr = (V *)c->d_scratch;
    PlainFFT<T> fft;
    fft.init(c);
    const Derived &d = c->dv;
    const int gN = blocks_for(n), gFN = blocks_for((int64_t)F * n);
    k_entry<T><<<gFN, kThreads, 0, st>>>(fld, (const V *)c->d_pump, n, F, c->cavity.resonant_mask,
                                          c->dv.ns, c->d_ctl);
    // every crystal in order; z of the e^{i dk z} factor restarts in each
    for (int i = 0; i < c->ncry; i++) {
        const CryDesc &cd = c->h_cry[i];
        const V *ekz = (const V *)cd.ekz;
        const T hc = (T)cd.h;
        const KerrG<T> G = kerr_g<T>(cd.kerr_g);
        for (int j = 0; j < cd.nz; j++) {
            for (int half = 0; half < 2; half++) {
                int q0 = 4 * j + 2 * half;
                if (F == 3)
                    k_rk4<T, 3><<<gN, kThreads, 0, st>>>(fld, n, ekz, q0, hc, (T)cd.kappa[0],
                                                         (T)cd.kappa[1], (T)cd.kappa[2],
                                                         cd.use_dk != 0, cd.kerr != 0, G);
                else
                    k_rk4<T, 2><<<gN, kThreads, 0, st>>>(fld, n, ekz, q0, hc, (T)cd.kappa[0],
                                                         (T)cd.kappa[1], (T)cd.kappa[2],
                                                         cd.use_dk != 0, cd.kerr != 0, G);
                if (half == 0) {
                    fft.template run<-1>(fld, scr, F, st);
                    k_mul_table<T><<<gFN, kThreads, 0, st>>>(fld, (const V *)cd.disp, F * n);
                    fft.template run<1>(fld, scr, F, st);
                }
            }
        }
    }
    k_power_sums<T><<<F, 512, 0, st>>>(fld, n, c->d_ctl);
    k_save_output<T><<<gFN, kThreads, 0, st>>>(fld, (V *)c->d_out, n, F, (T)d.outscale[0],
                                                (T)d.outscale[1], (T)d.outscale[2],
                                                (V *)c->d_hist, c->d_ctl);
    // cavity spectral visit: every resonant field with GDD or delay, and the
    // signal for its spectral centroid
    bool need_all = false;
    for (int x = 0; x < F; x++)
        if ((c->cavity.resonant_mask & (1u << x)) &&
            (c->cavity.gdd_s2[x] != 0.0 || c->cavity.delay_s != 0.0))
            need_all = true;
    V *sig = fld + (size_t)n;
    if (need_all) {
        fft.template run<-1>(fld, scr, F, st);
        k_spec_sums<T><<<1, 1024, 0, st>>>(sig, n, c->d_ctl);
        k_mul_table<T><<<gFN, kThreads, 0, st>>>(fld, (const V *)c->d_gdd, F * n);
        fft.template run<1>(fld, scr, F, st);
    } else {
        // centroid only: transform a copy of the signal
        V *copy = scr + (size_t)n; // second field slot of scratch
        cudaMemcpyAsync(copy, sig, (size_t)n * sizeof(V), cudaMemcpyDeviceToDevice, st);
        fft.template run<-1>(copy, scr, 1, st);
        k_spec_sums<T><<<1, 1024, 0, st>>>(copy, n, c->d_ctl);
    }
    CavArgs ca;
    for (int x = 0; x < 3; x++) {
        ca.bc_re[x] = d.bc_re[x];
        ca.bc_im[x] = d.bc_im[x];
    }
    ca.eom_beta = c->cavity.eom_beta_rad;
    ca.eom_f = c->cavity.eom_f_hz;
    ca.t_rt = c->cavity.t_rt_s > 0.0 ? c->cavity.t_rt_s : c->grid.t_window_s;
    ca.dt = c->grid.t_window_s / (double)n;
    ca.resmask = c->cavity.resonant_mask;
    ca.eom = d.eom ? 1 : 0;
    k_cavity_time<T><<<gN, kThreads, 0, st>>>(fld, n, F, ca, c->d_ctl);
    k_end_rt<<<1, 1, 0, st>>>(c->d_ctl);
    return cudaGetLastError() == cudaSuccess ? OPO_OK : OPO_E_CUDA;
}

template <class T>
void prepare()
{
    const int lim = 200 * 1024;
    cudaFuncSetAttribute(k_fft_cols<T, -1>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    cudaFuncSetAttribute(k_fft_cols<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    cudaFuncSetAttribute(k_fft_rows<T, -1>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    cudaFuncSetAttribute(k_fft_rows<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
}

} // namespace

void plain_prepare(opo_ctx *c)
{
    if (c->prec == OPO_FP64)
        prepare<double>();
    else
        prepare<float>();
}

int plain_enqueue_roundtrip(opo_ctx *c, cudaStream_t s)
{
    return c->prec == OPO_FP64 ? enqueue_rt<double>(c, s) : enqueue_rt<float>(c, s);
}

namespace {

// The crystal pass alone (nz symmetrized steps) on caller-provided buffers.
template <class T>
int pass_raw(void *fields, void *scratch, const void *tw, const void *disp, const void *ekz,
             int n, int F, int nz, const double kappa[3], double h, bool use_dk,
             const double *kg, cudaStream_t st)
{
    const double zero[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    const bool kerr = kg != nullptr;
    const KerrG<T> G = kerr_g<T>(kg ? kg : zero);
    using V = cv<T>;
    prepare<T>();
    V *fld = (V *)fields;
    V *scr = (V *)scratch;
    PlainFFT<T> fft;
    fft.init_raw(n, ilog2((unsigned)n), (const V *)tw);
    const int gN = blocks_for(n), gFN = blocks_for((int64_t)F * n);
    for (int j = 0; j < nz; j++) {
        for (int half = 0; half < 2; half++) {
            int q0 = 4 * j + 2 * half;
            if (F == 3)
                k_rk4<T, 3><<<gN, kThreads, 0, st>>>(fld, n, (const V *)ekz, q0, (T)h, (T)kappa[0],
                                                     (T)kappa[1], (T)kappa[2], use_dk, kerr, G);
            else
                k_rk4<T, 2><<<gN, kThreads, 0, st>>>(fld, n, (const V *)ekz, q0, (T)h, (T)kappa[0],
                                                     (T)kappa[1], (T)kappa[2], use_dk, kerr, G);
            if (half == 0) {
                fft.template run<-1>(fld, scr, F, st);
                k_mul_table<T><<<gFN, kThreads, 0, st>>>(fld, (const V *)disp, F * n);
                fft.template run<1>(fld, scr, F, st);
            }
        }
    }
    return cudaGetLastError() == cudaSuccess ? OPO_OK : OPO_E_CUDA;
}

} // namespace

int plain_pass_raw(void *fields, void *scratch, const void *tw, const void *disp, const void *ekz,
                   int n, int F, int nz, const double kappa[3], double h, bool use_dk,
                   const double *kerr_g, bool dbl, cudaStream_t st)
{
    return dbl ? pass_raw<double>(fields, scratch, tw, disp, ekz, n, F, nz, kappa, h, use_dk,
                                  kerr_g, st)
               : pass_raw<float>(fields, scratch, tw, disp, ekz, n, F, nz, kappa, h, use_dk,
                                 kerr_g, st);
}

} // namespace opo
