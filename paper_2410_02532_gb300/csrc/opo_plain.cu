// opo_plain.cu -- the plain GPU form of one OPO round trip: one kernel per
// operation per z-step (arXiv 2410.02532, Sec. 2.2 and the main loop of
// Sec. 4.1), with fields in HBM/L2 between kernels.  A round trip is
//   entry | nz x [RK4(dz/2), FFT, D, IFFT, RK4(dz/2)] | power sums |
//   output copy | FFT, signal spectrum sums, cavity spectral factor, IFFT |
//   mirror + EOM | round-trip counter
// and is captured once into a CUDA graph that every round trip replays.
//
// An FFT of a field that fits one CTA's shared memory (2^8 <= N <= 2^14 in
// FP32, 2^13 in FP64; N/32 or N/16 threads) is one kernel: the field is
// loaded once, every Stockham stage (radix 2..8) runs in place in shared
// memory, and it is stored once.  Larger fields (N = P Q) take two kernels (four-step
// decomposition, n = Q n1 + n2, k = k1 + P k2): P-point column transforms
// with the twiddle W_N^{n2 k1} written to scratch, then Q-point row
// transforms written back in natural order, each kernel transforming a batch
// of columns or rows in shared memory.
//
// Two launch forms share every kernel body: one instance per launch (a
// context's own graph; the allocation-free pass), and a batch in which each
// launch runs the same operation for every member, member blockIdx.z, with
// the member's pointers and parameters read from a device descriptor
// (PlainInst).  The paper's design is the first form; the second is that
// design over many instances at once.  Per element both do the same
// arithmetic, so a member advances bit for bit as it would alone.
#include <algorithm>
#include <type_traits>

#include "opo_common.cuh"
#include "opo_internal.h"

namespace opo {
namespace {

constexpr int kThreads = 256;

// ------------------------------------------------------------- bodies ----
// Each body works on one instance; elementwise bodies stride over
// blockIdx.x / gridDim.x.

// Round-trip entry: the input pump (table, or the ns-pulsed pump read at
// this round trip) replaces a non-resonant pump and is added to a resonant
// one; non-resonant signal/idler restart from zero.
template <class T>
__device__ __forceinline__ void entry_body(cv<T> *fields, const cv<T> *pump, int n, int F,
                                           unsigned resmask, const NsPump &ns, int64_t m)
{
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

// One RK4 step of h = dz/2 on every point (the nonlinear half step).  A
// thread takes two points per iteration (points j and j + stride, their
// loads issued together), and the grid is sized for a few iterations per
// thread: the step is short, so a thread's loads must be in flight together.
template <class T, int F>
__device__ __forceinline__ void rk4_body(cv<T> *fields, int n, const cv<T> *ekz, int q0, T h,
                                         const T *kap, bool use_e, bool kerr, const T *G)
{
    using V = cv<T>;
    const V one = cmk<V>((T)1, (T)0);
    const V e0 = use_e ? ekz[q0] : one, e1 = use_e ? ekz[q0 + 1] : one;
    const V e2 = use_e ? ekz[q0 + 2] : one;
    const int stride = gridDim.x * blockDim.x;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += 2 * stride) {
        const int j2 = j + stride;
        const bool two = j2 < n;
        V y[F], z[F];
#pragma unroll
        for (int x = 0; x < F; x++)
            y[x] = fields[(size_t)x * n + j];
        if (two) {
#pragma unroll
            for (int x = 0; x < F; x++)
                z[x] = fields[(size_t)x * n + j2];
        }
        if (kerr)
            rk4_point_kerr<F>(y, e0, e1, e2, kap, h, use_e, G);
        else
            rk4_point<F>(y, e0, e1, e2, kap, h, use_e);
#pragma unroll
        for (int x = 0; x < F; x++)
            fields[(size_t)x * n + j] = y[x];
        if (two) {
            if (kerr)
                rk4_point_kerr<F>(z, e0, e1, e2, kap, h, use_e, G);
            else
                rk4_point<F>(z, e0, e1, e2, kap, h, use_e);
#pragma unroll
            for (int x = 0; x < F; x++)
                fields[(size_t)x * n + j2] = z[x];
        }
    }
}

// Column pass of one field: loads columns n2 in [cb B, cb B + B) of
// src[Q n1 + n2], transforms over n1, multiplies W_N^{DIR n2 k1} and writes
// dst[k1 Q + n2].
template <class T, int DIR>
__device__ __forceinline__ void fft_cols_body(const cv<T> *__restrict__ src, cv<T> *__restrict__ dst,
                                              int n, int P, int Q, int logP, int logn, int B,
                                              const cv<T> *__restrict__ tw, int cb)
{
    using V = cv<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V *s0 = reinterpret_cast<V *>(smem_raw);
    V *s1 = s0 + B * P;
    const int n2b = cb * B;
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

// Row pass of one field: loads rows k1 in [rb B, rb B + B) of
// src[k1 Q + n2], transforms over n2 and writes dst[k1 + P k2].
template <class T, int DIR>
__device__ __forceinline__ void fft_rows_body(const cv<T> *__restrict__ src, cv<T> *__restrict__ dst,
                                              int n, int P, int Q, int logQ, int logn, int B,
                                              const cv<T> *__restrict__ tw, int rb)
{
    using V = cv<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int Lp = Q + 1; // padded row stride
    V *s0 = reinterpret_cast<V *>(smem_raw);
    V *s1 = s0 + B * Lp;
    const int k1b = rb * B;
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

// ---- whole-field transform (2^8 <= N <= 2^14 in FP32, 2^13 in FP64)
// The field sits in one CTA's shared memory and the transform runs as a few
// register passes of a Stockham FFT (butterfly j of a radix-R pass with
// stride Ns reads x[j + r N/R], multiplies by W_{Ns R}^{r k}, k = j mod Ns,
// takes an R-point DFT and writes output r at (j - k) R + k + r Ns): first
// one pass of the remaining radix 2^(log2 N mod 4) if there is one (Ns = 1:
// no twiddles), then radix-16 passes.  The first pass reads the field from
// global memory straight into registers and the last writes it back from
// registers, so shared memory holds only the intermediate passes (and the
// twiddle table).  N is a compile-time constant: every index is then a
// register plus an immediate.
// VPT values per thread (N/VPT threads): 32 in FP32 (two radix-16
// butterflies, up to 128 registers at 512 threads), 16 in FP64.
template <class T> constexpr int kFieldVpt = sizeof(T) == 8 ? 16 : 32;
template <class T> constexpr int kFieldThreads = 512;
template <class T> constexpr int kFieldMaxLog = sizeof(T) == 8 ? 13 : 14;
constexpr int kFieldMinLog = 8;

// shared memory: the field with one pad element after every 16 (index i at
// i + i/16, which spreads the stride-R stores over the banks)
__device__ __forceinline__ int fpad(int i) { return i + (i >> 4); }
// the half-wave twiddle table W_N^i, i < N/2, XOR-swizzled so that lanes
// reading W_N^{c k} at consecutive k mostly hit distinct banks
__device__ __forceinline__ int tsw(int i) { return i ^ (((i >> 4) ^ (i >> 8)) & 15); }

__host__ __device__ constexpr int field_lr(int logn, int p)
{
    return (logn % 4 != 0 && p == 0) ? logn % 4 : 4;
}
__host__ __device__ constexpr int field_npass(int logn) { return logn / 4 + (logn % 4 ? 1 : 0); }
__host__ __device__ constexpr int field_lns(int logn, int p)
{
    return p == 0 ? 0 : field_lns(logn, p - 1) + field_lr(logn, p - 1);
}
__host__ __device__ constexpr int field_smem_elems(int logn)
{
    return (1 << logn) + (1 << logn) / 16 + (1 << logn) / 2;
}

// Twiddles of a radix-16 pass for butterfly k: input r is multiplied by
// W_{16 Ns}^{r k} = W_N^e, e = r k 2^SH < N, each the table's own entry
// (W_N^{N/2 + i} = -W_N^i): no twiddle is formed from a product of others,
// whose rounding, repeated every z-step, shifts the long-run solution.
template <int LOGN, int SH, int DIR, class V>
__device__ __forceinline__ void field_twiddle16(V *v, const V *tab, int k)
{
    constexpr int HALF = (1 << (LOGN - 1)) - 1;
#pragma unroll
    for (int r = 1; r < 16; r++) {
        const int e = (r * k) << SH;
        V w = tab[tsw(e & HALF)];
        if (e >> (LOGN - 1)) {
            w.x = -w.x;
            w.y = -w.y;
        }
        if (DIR > 0)
            w.y = -w.y;
        v[r] = cmul(v[r], w);
    }
}

// Pass P of the transform; a is the field in global memory, s the padded
// shared copy, tab the swizzled quarter-wave table.
template <int LOGN, int P, int VPT, int DIR, class V>
__device__ __forceinline__ void field_pass(V *a, V *s, const V *tab)
{
    constexpr int N = 1 << LOGN, T = N / VPT;
    constexpr int LR = field_lr(LOGN, P), R = 1 << LR;
    constexpr int LNS = field_lns(LOGN, P), NS = 1 << LNS;
    constexpr int B = VPT / R; // butterflies per thread
    constexpr int LAST = field_npass(LOGN) - 1;
    constexpr int SH = LOGN - LNS - LR; // W_{Ns R} = W_N^{2^SH}
    static_assert(NS == 1 || R == 16, "only the first pass has a radix below 16");
    V v[B][R];
#pragma unroll
    for (int q = 0; q < B; q++) {
        const int j = (int)threadIdx.x + q * T;
#pragma unroll
        for (int r = 0; r < R; r++)
            v[q][r] = P == 0 ? a[j + r * (N / R)] : s[fpad(j + r * (N / R))];
        if constexpr (NS > 1)
            field_twiddle16<LOGN, SH, DIR>(v[q], tab, j & (NS - 1));
        dft<R, DIR>(v[q]);
    }
    if constexpr (P > 0 && P < LAST)
        __syncthreads(); // in place: every read of the pass before any write
#pragma unroll
    for (int q = 0; q < B; q++) {
        const int j = (int)threadIdx.x + q * T;
        const int k = j & (NS - 1);
        const int base = (j - k) * R + k;
#pragma unroll
        for (int r = 0; r < R; r++) {
            if constexpr (P == LAST)
                a[base + r * NS] = v[q][r];
            else
                s[fpad(base + r * NS)] = v[q][r];
        }
    }
    if constexpr (P < LAST)
        __syncthreads();
}

template <int LOGN, int P, int VPT, int DIR, class V>
__device__ __forceinline__ void field_passes(V *a, V *s, const V *tab)
{
    if constexpr (P < field_npass(LOGN)) {
        field_pass<LOGN, P, VPT, DIR>(a, s, tab);
        field_passes<LOGN, P + 1, VPT, DIR>(a, s, tab);
    }
}

// In-place transform of one field of 2^LOGN points (blockDim = N / VPT);
// tw is the global table W_N^i, i < N.
template <class T, int LOGN, int DIR>
__device__ __forceinline__ void fft_field_body(cv<T> *a, const cv<T> *__restrict__ tw)
{
    using V = cv<T>;
    constexpr int N = 1 << LOGN;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V *s = reinterpret_cast<V *>(smem_raw);
    V *tab = s + N + N / 16;
    for (int i = threadIdx.x; i < N / 2; i += blockDim.x)
        tab[tsw(i)] = tw[i];
    // the first pass needs no twiddles and writes s only after reading a;
    // its closing barrier publishes the table as well
    field_passes<LOGN, 0, kFieldVpt<T>, DIR>(a, s, tab);
}

// a[i] *= tab[i]: four elements blockDim apart per thread and iteration, so
// that each thread has eight loads in flight
template <class T>
__device__ __forceinline__ void mul_table_body(cv<T> *a, const cv<T> *__restrict__ tab, int total)
{
    constexpr int U = 4;
    const int bd = blockDim.x;
    for (int i = blockIdx.x * U * bd + threadIdx.x; i < total; i += gridDim.x * U * bd) {
        cv<T> x[U], t[U];
#pragma unroll
        for (int q = 0; q < U; q++) {
            if (i + q * bd < total) {
                x[q] = a[i + q * bd];
                t[q] = tab[i + q * bd];
            }
        }
#pragma unroll
        for (int q = 0; q < U; q++)
            if (i + q * bd < total)
                a[i + q * bd] = cmul(x[q], t[q]);
    }
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

// Sum |A_x|^2 of the post-crystal field x into the raw observable slot of
// this round trip; a non-finite sum sets the error word.
template <class T>
__device__ __forceinline__ void power_body(const cv<T> *fields, int n, int x, DevCtl *ctl)
{
    __shared__ double red[32];
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
__device__ __forceinline__ void spec_body(const cv<T> *spec, int n, DevCtl *ctl)
{
    __shared__ double red[32];
    double s0 = 0.0, s1 = 0.0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        double p = (double)cabs2(spec[k]);
        int kk = (k < n / 2) ? k : k - n;
        s0 += p;
        s1 = __fma_rn((double)kk, p, s1);
    }
    s0 = block_sum(s0, red);
    s1 = block_sum(s1, red);
    if (threadIdx.x == 0) {
        ctl->obs[ctl->slot * kNslot + 3] = s0;
        ctl->obs[ctl->slot * kNslot + 4] = s1;
    }
}

// Output-coupled fields (and their history row) of this round trip.
template <class T>
__device__ __forceinline__ void save_body(const cv<T> *fields, cv<T> *out, int n, int F,
                                          const T *sc, cv<T> *hist, const DevCtl *ctl)
{
    cv<T> *row = hist ? hist + (size_t)ctl->slot * F * n : nullptr; // history row of this round trip
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < F * n; i += gridDim.x * blockDim.x) {
        const cv<T> o = cscale(fields[i], sc[i / n]);
        out[i] = o;
        if (row)
            row[i] = o;
    }
}

// Mirror sqrt(R) e^{i delta} (Eq. (BC)) then the EOM phase (Sec. 2.3 item 2)
// on resonant fields; the EOM argument frac(f_pm (tau_n + m t_rt)) is formed
// in FP64.
template <class T>
__device__ __forceinline__ void cavity_body(cv<T> *fields, int n, int F, const PlainCav &a,
                                            int64_t m)
{
    using V = cv<T>;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        V mod = cmk<V>((T)1, (T)0);
        if (a.eom) {
            const double u = __fma_rn(a.eom_f, (double)(j - n / 2) * a.dt,
                                      a.eom_f * ((double)m * a.t_rt));
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

// ------------------------------------------- single-instance kernels ----

template <class T>
__global__ void k_entry(cv<T> *fields, const cv<T> *pump, int n, int F, unsigned resmask,
                        NsPump ns, const DevCtl *ctl)
{
    entry_body<T>(fields, pump, n, F, resmask, ns, ctl->rt0 + ctl->slot);
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
    const T kap[3] = {k0, k1, k2};
    rk4_body<T, F>(fields, n, ekz, q0, h, kap, use_e, kerr, G.g);
}

// grid (Q/B, fields)
template <class T, int DIR>
__global__ void k_fft_cols(const cv<T> *__restrict__ in, cv<T> *__restrict__ out, int n, int P,
                           int Q, int logP, int logn, int B, const cv<T> *__restrict__ tw)
{
    fft_cols_body<T, DIR>(in + (size_t)blockIdx.y * n, out + (size_t)blockIdx.y * n, n, P, Q, logP,
                          logn, B, tw, blockIdx.x);
}

// grid (P/B, fields)
template <class T, int DIR>
__global__ void k_fft_rows(const cv<T> *__restrict__ in, cv<T> *__restrict__ out, int n, int P,
                           int Q, int logQ, int logn, int B, const cv<T> *__restrict__ tw)
{
    fft_rows_body<T, DIR>(in + (size_t)blockIdx.y * n, out + (size_t)blockIdx.y * n, n, P, Q, logQ,
                          logn, B, tw, blockIdx.x);
}

// grid (fields): one whole-field transform per CTA, in place
template <class T, int LOGN, int DIR>
__global__ void __launch_bounds__(kFieldThreads<T>, 1)
    k_fft_field(cv<T> *a, const cv<T> *__restrict__ tw)
{
    fft_field_body<T, LOGN, DIR>(a + ((size_t)blockIdx.y << LOGN), tw);
}

template <class T>
__global__ void k_mul_table(cv<T> *a, const cv<T> *__restrict__ tab, int total)
{
    mul_table_body<T>(a, tab, total);
}

// one block per field
template <class T>
__global__ void k_power_sums(const cv<T> *fields, int n, DevCtl *ctl)
{
    power_body<T>(fields, n, blockIdx.x, ctl);
}

template <class T>
__global__ void k_spec_sums(const cv<T> *spec, int n, DevCtl *ctl)
{
    spec_body<T>(spec, n, ctl);
}

template <class T>
__global__ void k_save_output(const cv<T> *fields, cv<T> *out, int n, int F, T s0, T s1, T s2,
                              cv<T> *hist, const DevCtl *ctl)
{
    const T sc[3] = {s0, s1, s2};
    save_body<T>(fields, out, n, F, sc, hist, ctl);
}

template <class T>
__global__ void k_cavity_time(cv<T> *fields, int n, int F, PlainCav a, const DevCtl *ctl)
{
    cavity_body<T>(fields, n, F, a, ctl->rt0 + ctl->slot);
}

__global__ void k_end_rt(DevCtl *ctl)
{
    ctl->slot += 1;
}

// --------------------------------------------------- batch kernels ----
// Member blockIdx.z; the member's pointers and parameters come from its
// descriptor.  Kernels of the cavity visit (mode argument of the transforms)
// act on every field where the member's visit transforms every field
// (spec_all), else on a copy of its signal in scratch slot 1.

template <class T>
__global__ void kb_entry(const PlainInst *__restrict__ insts, int n, int F)
{
    const PlainInst &I = insts[blockIdx.z];
    entry_body<T>((cv<T> *)I.fields, (const cv<T> *)I.pump, n, F, I.cav.resmask, I.ns,
                  I.ctl->rt0 + I.ctl->slot);
}

template <class T, int F>
__global__ void kb_rk4(const PlainInst *__restrict__ insts, int n, int kc, int q0)
{
    const PlainInst &I = insts[blockIdx.z];
    const CryDesc &cd = I.cry[kc];
    // the crystal's constants in the field precision (FP32: the copies the
    // host rounded; a conversion from double on the device issues on the
    // FP64 pipe, a small fraction of the FP32 rate, and per thread these
    // conversions outweighed the step itself)
    T sc[13];
#pragma unroll
    for (int i = 0; i < 13; i++) {
        if constexpr (sizeof(T) == 4)
            sc[i] = cd.kf[i];
        else
            sc[i] = i < 3 ? cd.kappa[i] : i == 3 ? cd.h : cd.kerr_g[i - 4];
    }
    const T kap[3] = {sc[0], sc[1], sc[2]};
    T G[9];
#pragma unroll
    for (int i = 0; i < 9; i++)
        G[i] = sc[4 + i];
    rk4_body<T, F>((cv<T> *)I.fields, n, (const cv<T> *)cd.ekz, q0, sc[3], kap, cd.use_dk != 0,
                   cd.kerr != 0, G);
}

// The buffer a transform of mode `mode` works on and its field count:
// 0 the fields (all F); 1 the forward cavity visit (the fields, or the signal
// copy); 2 the inverse cavity visit (the fields where spec_all, else none).
template <class T>
__device__ __forceinline__ cv<T> *visit_buffer(const PlainInst &I, int mode, int n, int F,
                                               int *count)
{
    if (mode == 0 || (mode == 2 && I.spec_all)) {
        *count = F;
        return (cv<T> *)I.fields;
    }
    if (mode == 1) {
        *count = I.spec_all ? F : 1;
        return I.spec_all ? (cv<T> *)I.fields : (cv<T> *)I.scratch + n;
    }
    *count = 0;
    return nullptr;
}

// grid (Q/B, F, members); the column pass writes scratch
template <class T, int DIR>
__global__ void kb_fft_cols(const PlainInst *__restrict__ insts, int mode, int n, int F, int P,
                            int Q, int logP, int logn, int B)
{
    const PlainInst &I = insts[blockIdx.z];
    int count;
    const cv<T> *a = visit_buffer<T>(I, mode, n, F, &count);
    if ((int)blockIdx.y >= count)
        return;
    fft_cols_body<T, DIR>(a + (size_t)blockIdx.y * n, (cv<T> *)I.scratch + (size_t)blockIdx.y * n,
                          n, P, Q, logP, logn, B, (const cv<T> *)I.tw, blockIdx.x);
}

// grid (P/B, F, members); the row pass reads scratch
template <class T, int DIR>
__global__ void kb_fft_rows(const PlainInst *__restrict__ insts, int mode, int n, int F, int P,
                            int Q, int logQ, int logn, int B)
{
    const PlainInst &I = insts[blockIdx.z];
    int count;
    cv<T> *a = visit_buffer<T>(I, mode, n, F, &count);
    if ((int)blockIdx.y >= count)
        return;
    fft_rows_body<T, DIR>((const cv<T> *)I.scratch + (size_t)blockIdx.y * n, a + (size_t)blockIdx.y * n,
                          n, P, Q, logQ, logn, B, (const cv<T> *)I.tw, blockIdx.x);
}

// grid (1, F, members): whole-field transforms of the buffer of `mode`
template <class T, int LOGN, int DIR>
__global__ void __launch_bounds__(kFieldThreads<T>, 1)
    kb_fft_field(const PlainInst *__restrict__ insts, int mode, int F)
{
    const PlainInst &I = insts[blockIdx.z];
    int count;
    cv<T> *a = visit_buffer<T>(I, mode, 1 << LOGN, F, &count);
    if ((int)blockIdx.y >= count)
        return;
    fft_field_body<T, LOGN, DIR>(a + ((size_t)blockIdx.y << LOGN), (const cv<T> *)I.tw);
}

// f(std::integral_constant<int, L>{}) for the whole-field size L = log2 N
template <class T, class Fn>
void with_field_log(int logn, Fn &&f)
{
    using std::integral_constant;
    switch (logn) {
    case 8: f(integral_constant<int, 8>{}); break;
    case 9: f(integral_constant<int, 9>{}); break;
    case 10: f(integral_constant<int, 10>{}); break;
    case 11: f(integral_constant<int, 11>{}); break;
    case 12: f(integral_constant<int, 12>{}); break;
    case 13: f(integral_constant<int, 13>{}); break;
    case 14:
        if constexpr (kFieldMaxLog<T> >= 14)
            f(integral_constant<int, 14>{});
        break;
    default: break;
    }
}

// kc >= 0: dispersion factors of crystal kc; kc < 0: the cavity spectral
// factors (members whose visit transforms every field)
template <class T>
__global__ void kb_mul_table(const PlainInst *__restrict__ insts, int n, int F, int kc)
{
    const PlainInst &I = insts[blockIdx.z];
    if (kc < 0 && !I.spec_all)
        return;
    const cv<T> *tab = (const cv<T> *)(kc >= 0 ? I.cry[kc].disp : I.gdd);
    mul_table_body<T>((cv<T> *)I.fields, tab, F * n);
}

// grid (F, 1, members)
template <class T>
__global__ void kb_power_sums(const PlainInst *__restrict__ insts, int n)
{
    const PlainInst &I = insts[blockIdx.z];
    power_body<T>((const cv<T> *)I.fields, n, blockIdx.x, I.ctl);
}

// the signal into scratch slot 1 where the visit transforms a copy
template <class T>
__global__ void kb_copy_signal(const PlainInst *__restrict__ insts, int n)
{
    const PlainInst &I = insts[blockIdx.z];
    if (I.spec_all)
        return;
    const cv<T> *src = (const cv<T> *)I.fields + n;
    cv<T> *dst = (cv<T> *)I.scratch + n;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x)
        dst[j] = src[j];
}

template <class T>
__global__ void kb_spec_sums(const PlainInst *__restrict__ insts, int n)
{
    const PlainInst &I = insts[blockIdx.z];
    const cv<T> *spec = I.spec_all ? (const cv<T> *)I.fields + n : (const cv<T> *)I.scratch + n;
    spec_body<T>(spec, n, I.ctl);
}

template <class T>
__global__ void kb_save_output(const PlainInst *__restrict__ insts, int n, int F)
{
    const PlainInst &I = insts[blockIdx.z];
    const T sc[3] = {(T)I.outscale[0], (T)I.outscale[1], (T)I.outscale[2]};
    save_body<T>((const cv<T> *)I.fields, (cv<T> *)I.out, n, F, sc, (cv<T> *)I.hist, I.ctl);
}

template <class T>
__global__ void kb_cavity_time(const PlainInst *__restrict__ insts, int n, int F)
{
    const PlainInst &I = insts[blockIdx.z];
    cavity_body<T>((cv<T> *)I.fields, n, F, I.cav, I.ctl->rt0 + I.ctl->slot);
}

__global__ void kb_end_rt(const PlainInst *__restrict__ insts, int count)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x)
        insts[i].ctl->slot += 1;
}

__global__ void kb_begin(const PlainCall *__restrict__ calls, int count)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
        const PlainCall &c = calls[i];
        c.ctl->rt0 = c.rt0;
        c.ctl->slot = 0;
        c.ctl->obs = c.obs;
        c.ctl->parts = 1;
    }
}

// The trace rows of every member (the arithmetic of the single-instance
// finalize with one partial sum per round trip).
__global__ void kb_finalize(const PlainCall *__restrict__ calls, int count, int64_t M)
{
    const int64_t total = (int64_t)count * M;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const PlainCall &c = calls[t / M];
        const int64_t s = t % M;
        double sum[kNslot] = {0, 0, 0, 0, 0};
        for (int q = 0; q < kNslot; q++)
            sum[q] += c.obs[s * kNslot + q];
        for (int x = 0; x < 3; x++)
            c.trace[s * 4 + x] = (x < c.F) ? sum[x] * c.inv_n * c.outscale2[x] * c.pscale[x] : 0.0;
        c.trace[s * 4 + 3] = sum[3] > 0.0 ? (sum[4] / sum[3]) / c.t_window : 0.0;
    }
}

int blocks_for(int64_t work)
{
    int64_t b = (work + kThreads - 1) / kThreads;
    return (int)(b < 1 ? 1 : (b > 1184 ? 1184 : b));
}

// FFT plan of length N: a field of N <= 2^14 (FP32) or 2^13 (FP64) points,
// and at least 2^8, is transformed whole in one CTA (one kernel, N/VPT
// threads, the field in shared memory); larger fields as N = P Q in two
// kernels (column pass, row pass) with their batch sizes and shared memory.
struct FFTShape {
    int n, logn, P, Q, logP, logQ, Bc, Br;
    size_t smc, smr;
    bool whole;       // one kernel per transform
    size_t smf;       // its shared memory (the padded field, twiddle tables)
    int vpt;          // its values per thread (N/vpt threads)
    template <class T>
    void init(int n_)
    {
        n = n_;
        logn = ilog2((unsigned)n);
        whole = logn >= kFieldMinLog && logn <= kFieldMaxLog<T>;
        smf = whole ? (size_t)field_smem_elems(logn) * sizeof(cv<T>) : 0;
        vpt = kFieldVpt<T>;
        logP = logn / 2;
        logQ = logn - logP;
        P = 1 << logP;
        Q = 1 << logQ;
        int seg = (sizeof(T) == 8) ? 4 : 8; // 64-byte column segments
        Bc = Q < seg ? Q : seg;
        Br = P < seg ? P : seg;
        smc = (size_t)2 * Bc * P * sizeof(cv<T>);
        smr = (size_t)2 * Br * (Q + 1) * sizeof(cv<T>);
    }
};

template <class T>
struct PlainFFT {
    FFTShape sh{};
    const cv<T> *tw;
    void init_raw(int n_, const cv<T> *tw_)
    {
        sh.template init<T>(n_);
        tw = tw_;
    }
    // transform `count` consecutive fields of `a` in place, scratch `s`
    template <int DIR>
    void run(cv<T> *a, cv<T> *s, int count, cudaStream_t st) const
    {
        if (sh.whole) {
            const cv<T> *t = tw;
            const int threads = sh.n / sh.vpt;
            const size_t sm = sh.smf;
            with_field_log<T>(sh.logn, [&](auto L) {
                k_fft_field<T, decltype(L)::value, DIR><<<dim3(1, count), threads, sm, st>>>(a, t);
            });
            return;
        }
        dim3 gc(sh.Q / sh.Bc, count), gr(sh.P / sh.Br, count);
        k_fft_cols<T, DIR><<<gc, kThreads, sh.smc, st>>>(a, s, sh.n, sh.P, sh.Q, sh.logP, sh.logn,
                                                          sh.Bc, tw);
        k_fft_rows<T, DIR><<<gr, kThreads, sh.smr, st>>>(s, a, sh.n, sh.P, sh.Q, sh.logQ, sh.logn,
                                                          sh.Br, tw);
    }
};

PlainCav plain_cav(const opo_ctx *c)
{
    PlainCav ca;
    for (int x = 0; x < 3; x++) {
        ca.bc_re[x] = c->dv.bc_re[x];
        ca.bc_im[x] = c->dv.bc_im[x];
    }
    ca.eom_beta = c->cavity.eom_beta_rad;
    ca.eom_f = c->cavity.eom_f_hz;
    ca.t_rt = c->cavity.t_rt_s > 0.0 ? c->cavity.t_rt_s : c->grid.t_window_s;
    ca.dt = c->grid.t_window_s / (double)c->n;
    ca.resmask = c->cavity.resonant_mask;
    ca.eom = c->dv.eom ? 1 : 0;
    return ca;
}

// The cavity visit transforms every field when a resonant field has GDD or
// the timing mismatch is on; otherwise only a copy of the signal (for its
// spectral centroid).
bool spec_all_fields(const opo_ctx *c)
{
    for (int x = 0; x < c->F; x++)
        if ((c->cavity.resonant_mask & (1u << x)) &&
            (c->cavity.gdd_s2[x] != 0.0 || c->cavity.delay_s != 0.0))
            return true;
    return false;
}

template <class T>
int enqueue_rt(opo_ctx *c, cudaStream_t st)
{
    using V = cv<T>;
    const int n = c->n, F = c->F;
    V *fld = (V *)c->d_fields;
    V *scr = (V *)c->d_scratch;
    PlainFFT<T> fft;
    fft.init_raw(n, (const V *)c->d_tw);
    const Derived &d = c->dv;
    const int gN = blocks_for(n), gFN = blocks_for((int64_t)F * n);
    const int gM = blocks_for(((int64_t)F * n + 7) / 8); // mul_table: 8 elements a thread
    const int gR = blocks_for(((int64_t)n + 3) / 4);     // rk4: 4 points a thread
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
                    k_rk4<T, 3><<<gR, kThreads, 0, st>>>(fld, n, ekz, q0, hc, (T)cd.kappa[0],
                                                         (T)cd.kappa[1], (T)cd.kappa[2],
                                                         cd.use_dk != 0, cd.kerr != 0, G);
                else
                    k_rk4<T, 2><<<gR, kThreads, 0, st>>>(fld, n, ekz, q0, hc, (T)cd.kappa[0],
                                                         (T)cd.kappa[1], (T)cd.kappa[2],
                                                         cd.use_dk != 0, cd.kerr != 0, G);
                if (half == 0) {
                    fft.template run<-1>(fld, scr, F, st);
                    k_mul_table<T><<<gM, kThreads, 0, st>>>(fld, (const V *)cd.disp, F * n);
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
    V *sig = fld + (size_t)n;
    if (spec_all_fields(c)) {
        fft.template run<-1>(fld, scr, F, st);
        k_spec_sums<T><<<1, 1024, 0, st>>>(sig, n, c->d_ctl);
        k_mul_table<T><<<gM, kThreads, 0, st>>>(fld, (const V *)c->d_gdd, F * n);
        fft.template run<1>(fld, scr, F, st);
    } else {
        // centroid only: transform a copy of the signal
        V *copy = scr + (size_t)n; // second field slot of scratch
        cudaMemcpyAsync(copy, sig, (size_t)n * sizeof(V), cudaMemcpyDeviceToDevice, st);
        fft.template run<-1>(copy, scr, 1, st);
        k_spec_sums<T><<<1, 1024, 0, st>>>(copy, n, c->d_ctl);
    }
    k_cavity_time<T><<<gN, kThreads, 0, st>>>(fld, n, F, plain_cav(c), c->d_ctl);
    k_end_rt<<<1, 1, 0, st>>>(c->d_ctl);
    return cudaGetLastError() == cudaSuccess ? OPO_OK : OPO_E_CUDA;
}

// One round trip of every member of a batch, one launch per operation.
template <class T>
int enqueue_rt_batch(const opo_ctx *c0, const PlainInst *I, int count, cudaStream_t st)
{
    const int n = c0->n, F = c0->F;
    FFTShape sh{};
    sh.template init<T>(n);
    const int gN = blocks_for(n), gFN = blocks_for((int64_t)F * n);
    const int gM = blocks_for(((int64_t)F * n + 7) / 8); // mul_table: 8 elements a thread
    const int gR = blocks_for(((int64_t)n + 3) / 4);     // rk4: 4 points a thread
    auto fft = [&](int dir, int mode) {
        if (sh.whole) {
            const dim3 gf(1, F, count);
            with_field_log<T>(sh.logn, [&](auto L) {
                constexpr int LG = decltype(L)::value;
                if (dir < 0)
                    kb_fft_field<T, LG, -1><<<gf, sh.n / sh.vpt, sh.smf, st>>>(I, mode, F);
                else
                    kb_fft_field<T, LG, 1><<<gf, sh.n / sh.vpt, sh.smf, st>>>(I, mode, F);
            });
            return;
        }
        dim3 gc(sh.Q / sh.Bc, F, count), gr(sh.P / sh.Br, F, count);
        if (dir < 0) {
            kb_fft_cols<T, -1><<<gc, kThreads, sh.smc, st>>>(I, mode, n, F, sh.P, sh.Q, sh.logP,
                                                              sh.logn, sh.Bc);
            kb_fft_rows<T, -1><<<gr, kThreads, sh.smr, st>>>(I, mode, n, F, sh.P, sh.Q, sh.logQ,
                                                              sh.logn, sh.Br);
        } else {
            kb_fft_cols<T, 1><<<gc, kThreads, sh.smc, st>>>(I, mode, n, F, sh.P, sh.Q, sh.logP,
                                                             sh.logn, sh.Bc);
            kb_fft_rows<T, 1><<<gr, kThreads, sh.smr, st>>>(I, mode, n, F, sh.P, sh.Q, sh.logQ,
                                                             sh.logn, sh.Br);
        }
    };
    kb_entry<T><<<dim3(gFN, 1, count), kThreads, 0, st>>>(I, n, F);
    for (int i = 0; i < c0->ncry; i++) {
        for (int j = 0; j < c0->cry[i].nz; j++) {
            for (int half = 0; half < 2; half++) {
                const int q0 = 4 * j + 2 * half;
                if (F == 3)
                    kb_rk4<T, 3><<<dim3(gR, 1, count), kThreads, 0, st>>>(I, n, i, q0);
                else
                    kb_rk4<T, 2><<<dim3(gR, 1, count), kThreads, 0, st>>>(I, n, i, q0);
                if (half == 0) {
                    fft(-1, 0);
                    kb_mul_table<T><<<dim3(gM, 1, count), kThreads, 0, st>>>(I, n, F, i);
                    fft(1, 0);
                }
            }
        }
    }
    kb_power_sums<T><<<dim3(F, 1, count), 512, 0, st>>>(I, n);
    kb_save_output<T><<<dim3(gFN, 1, count), kThreads, 0, st>>>(I, n, F);
    kb_copy_signal<T><<<dim3(gN, 1, count), kThreads, 0, st>>>(I, n);
    fft(-1, 1);
    kb_spec_sums<T><<<dim3(1, 1, count), 1024, 0, st>>>(I, n);
    kb_mul_table<T><<<dim3(gM, 1, count), kThreads, 0, st>>>(I, n, F, -1);
    fft(1, 2);
    kb_cavity_time<T><<<dim3(gN, 1, count), kThreads, 0, st>>>(I, n, F);
    kb_end_rt<<<(count + 255) / 256, 256, 0, st>>>(I, count);
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
    cudaFuncSetAttribute(kb_fft_cols<T, -1>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    cudaFuncSetAttribute(kb_fft_cols<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    cudaFuncSetAttribute(kb_fft_rows<T, -1>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    cudaFuncSetAttribute(kb_fft_rows<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    for (int lg = kFieldMinLog; lg <= kFieldMaxLog<T>; lg++) {
        with_field_log<T>(lg, [&](auto L) {
            constexpr int LG = decltype(L)::value;
            const int sm = (int)(field_smem_elems(LG) * sizeof(cv<T>));
            cudaFuncSetAttribute(k_fft_field<T, LG, -1>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
            cudaFuncSetAttribute(k_fft_field<T, LG, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
            cudaFuncSetAttribute(kb_fft_field<T, LG, -1>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
            cudaFuncSetAttribute(kb_fft_field<T, LG, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
        });
    }
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

void plain_fill_inst(PlainInst &p, const opo_ctx *c)
{
    p = PlainInst{};
    p.fields = c->d_fields;
    p.out = c->d_out;
    p.scratch = c->d_scratch;
    p.hist = c->d_hist;
    p.pump = c->d_pump;
    p.gdd = c->d_gdd;
    p.tw = c->d_tw;
    p.cry = c->d_cry;
    p.ctl = c->d_ctl;
    p.ns = c->dv.ns;
    p.cav = plain_cav(c);
    for (int x = 0; x < 3; x++)
        p.outscale[x] = c->dv.outscale[x];
    p.spec_all = spec_all_fields(c) ? 1 : 0;
}

void plain_fill_call(PlainCall &p, const opo_ctx *c)
{
    p = PlainCall{};
    p.ctl = c->d_ctl;
    p.obs = c->d_obs;
    p.trace = c->d_trace;
    p.rt0 = c->rt;
    for (int x = 0; x < 3; x++) {
        p.outscale2[x] = c->dv.outscale[x] * c->dv.outscale[x];
        p.pscale[x] = c->dv.pscale[x];
    }
    p.inv_n = 1.0 / (double)c->n;
    p.t_window = c->grid.t_window_s;
    p.F = c->F;
}

int plain_batch_enqueue_roundtrip(const opo_ctx *c0, const PlainInst *d_insts, int count,
                                  cudaStream_t s)
{
    if (c0->prec == OPO_FP64) {
        prepare<double>();
        return enqueue_rt_batch<double>(c0, d_insts, count, s);
    }
    prepare<float>();
    return enqueue_rt_batch<float>(c0, d_insts, count, s);
}

int plain_batch_begin(const PlainCall *d_calls, int count, cudaStream_t s)
{
    kb_begin<<<(count + 255) / 256, 256, 0, s>>>(d_calls, count);
    return cudaGetLastError() == cudaSuccess ? OPO_OK : OPO_E_CUDA;
}

int plain_batch_finalize(const PlainCall *d_calls, int count, int64_t M, cudaStream_t s)
{
    if (M <= 0)
        return OPO_OK;
    const int64_t work = (int64_t)count * M;
    const int nb = (int)std::min<int64_t>((work + 255) / 256, 4096);
    kb_finalize<<<nb, 256, 0, s>>>(d_calls, count, M);
    return cudaGetLastError() == cudaSuccess ? OPO_OK : OPO_E_CUDA;
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
    fft.init_raw(n, (const V *)tw);
    const int gN = blocks_for(n), gFN = blocks_for((int64_t)F * n);
    const int gM = blocks_for(((int64_t)F * n + 7) / 8); // mul_table: 8 elements a thread
    const int gR = blocks_for(((int64_t)n + 3) / 4);     // rk4: 4 points a thread
    for (int j = 0; j < nz; j++) {
        for (int half = 0; half < 2; half++) {
            int q0 = 4 * j + 2 * half;
            if (F == 3)
                k_rk4<T, 3><<<gR, kThreads, 0, st>>>(fld, n, (const V *)ekz, q0, (T)h, (T)kappa[0],
                                                     (T)kappa[1], (T)kappa[2], use_dk, kerr, G);
            else
                k_rk4<T, 2><<<gR, kThreads, 0, st>>>(fld, n, (const V *)ekz, q0, (T)h, (T)kappa[0],
                                                     (T)kappa[1], (T)kappa[2], use_dk, kerr, G);
            if (half == 0) {
                fft.template run<-1>(fld, scr, F, st);
                k_mul_table<T><<<gM, kThreads, 0, st>>>(fld, (const V *)disp, F * n);
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
