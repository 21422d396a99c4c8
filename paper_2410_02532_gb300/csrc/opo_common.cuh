// opo_common.cuh -- device building blocks shared by the plain and fused
// split-step kernels: complex arithmetic on float2/double2, in-register DFTs
// of radix 2..16, the radix plan of a Stockham FFT, and the nonlinear RK4
// step of the coupled-wave equations (arXiv 2410.02532, Sec. 2.1 Eqs.
// (CEp)-(CEi); Sec. 2.2 RK4 for the nonlinear half steps).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

// ------------------------------------------------------------ complex ----

template <class T> struct cvec;
template <> struct cvec<float> { using type = float2; };
template <> struct cvec<double> { using type = double2; };
template <class T> using cv = typename cvec<T>::type;

template <class V> struct cscal;
template <> struct cscal<float2> { using type = float; };
template <> struct cscal<double2> { using type = double; };

template <class V>
__host__ __device__ __forceinline__ V cmk(typename cscal<V>::type re, typename cscal<V>::type im)
{
    V r;
    r.x = re;
    r.y = im;
    return r;
}
template <class V> __device__ __forceinline__ V cadd(V a, V b) { return cmk<V>(a.x + b.x, a.y + b.y); }
template <class V> __device__ __forceinline__ V csub(V a, V b) { return cmk<V>(a.x - b.x, a.y - b.y); }
// Fused multiply-add with the rounding fixed in the source: a sum of two
// products a b + c d can be contracted two ways, and the compiler may choose
// differently in two inlined copies of the same arithmetic; spelling the
// fma out makes every copy (first or later round trip of a launch, last step
// of a crystal, one or many instances) round the same.
__device__ __forceinline__ float fmad_(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fmad_(double a, double b, double c) { return __fma_rn(a, b, c); }
template <class V> __device__ __forceinline__ V cmul(V a, V b)
{
    return cmk<V>(fmad_(a.x, b.x, -(a.y * b.y)), fmad_(a.x, b.y, a.y * b.x));
}
// a * conj(b)
template <class V> __device__ __forceinline__ V cmulc(V a, V b)
{
    return cmk<V>(fmad_(a.x, b.x, a.y * b.y), fmad_(a.y, b.x, -(a.x * b.y)));
}
template <class V> __device__ __forceinline__ V cconj(V a) { return cmk<V>(a.x, -a.y); }
template <class V> __device__ __forceinline__ V cscale(V a, typename cscal<V>::type s)
{
    return cmk<V>(a.x * s, a.y * s);
}
// i * a
template <class V> __device__ __forceinline__ V cmuli(V a) { return cmk<V>(-a.y, a.x); }
template <class V> __device__ __forceinline__ typename cscal<V>::type cabs2(V a)
{
    return fmad_(a.x, a.x, a.y * a.y);
}

// ------------------------------------------------- in-register DFTs ----
// DFT of R values in natural order (R = 1 .. 32), X_k = sum_j v_j
// e^{DIR 2 pi i jk/R}, DIR = -1 forward, +1 inverse (unnormalized).
// Recursive even/odd split (radix-2 decimation in time); the constant
// twiddles are e^{DIR 2 pi i a/32}.

template <int A, int DIR, class V>
__device__ __forceinline__ V rot32(V x)
{
    // cos and sin of 2 pi a / 32, a = 0..15 (mathematical constants)
    constexpr double c32[16] = {1.00000000000000000000, 0.980785280403230449126, 0.923879532511286756128, 0.831469612302545237079,
                                0.707106781186547524401, 0.555570233019602224743, 0.382683432365089771728, 0.195090322016128267848,
                                0.0, -0.195090322016128267848, -0.382683432365089771728, -0.555570233019602224743,
                                -0.707106781186547524401, -0.831469612302545237079, -0.923879532511286756128, -0.980785280403230449126};
    constexpr double s32[16] = {0.0, 0.195090322016128267848, 0.382683432365089771728, 0.555570233019602224743,
                                0.707106781186547524401, 0.831469612302545237079, 0.923879532511286756128, 0.980785280403230449126,
                                1.00000000000000000000, 0.980785280403230449126, 0.923879532511286756128, 0.831469612302545237079,
                                0.707106781186547524401, 0.555570233019602224743, 0.382683432365089771728, 0.195090322016128267848};
    // Single precision: the nearest floats of cos and sin give every one of
    // these rotations a modulus below 1 (by 1.5e-8 to 5.8e-8 in |w|^2), so
    // every butterfly of every in-register DFT loses a little energy, the
    // same bins every z-step: over thousands of round trips that pulled the
    // FP32 steady state ~7e-4 below the FP64 one (P_s,out after 20000 round
    // trips of the 2^14 workload; 1.3e-4 fused and 4e-6 plain with these).  These pairs lie within
    // two units in the last place of the nearest floats (phase error below
    // 1e-7 rad) and are chosen so that each pair (a, 16 - a), which every
    // DFT uses equally often, has moduli errors of opposite sign: their sum
    // is below 1.6e-8 for every radix (nearest floats: -6.9e-8 at radix 8,
    // -3.0e-7 at 16, -5.9e-7 at 32).
    constexpr float c32f[16] = {1.0f, 0.98078531f, 0.923879564f, 0.831469595f, 0.707106769f,
                                0.555570245f, 0.382683486f, 0.195090353f, 0.0f, -0.195090294f,
                                -0.382683367f, -0.555570185f, -0.707106769f, -0.831469655f,
                                -0.923879504f, -0.980785251f};
    constexpr float s32f[16] = {0.0f, 0.195090294f, 0.382683367f, 0.555570245f, 0.707106769f,
                                0.831469595f, 0.923879504f, 0.980785251f, 1.0f, 0.98078531f,
                                0.923879564f, 0.831469655f, 0.707106829f, 0.555570185f,
                                0.382683486f, 0.195090353f};
    using S = typename cscal<V>::type;
    if constexpr (A == 0) {
        return x;
    } else if constexpr (A == 8) {
        return DIR < 0 ? cmk<V>(x.y, -x.x) : cmk<V>(-x.y, x.x);
    } else {
        const S c = sizeof(S) == 4 ? (S)c32f[A] : (S)c32[A];
        const S s = sizeof(S) == 4 ? (S)(DIR * s32f[A]) : (S)(DIR * s32[A]);
        return cmk<V>(fmad_(x.x, c, -(x.y * s)), fmad_(x.x, s, x.y * c));
    }
}

template <int R, int DIR, int K, class V>
__device__ __forceinline__ void dft_combine(V *v, const V *e, const V *o)
{
    if constexpr (K < R / 2) {
        V t = rot32<K * (32 / R), DIR>(o[K]);
        v[K] = cadd(e[K], t);
        v[K + R / 2] = csub(e[K], t);
        dft_combine<R, DIR, K + 1>(v, e, o);
    }
}

template <int R, int DIR, class V>
__device__ __forceinline__ void dft(V *v)
{
    if constexpr (R == 1) {
        return;
    } else if constexpr (R == 2) {
        V a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    } else {
        V e[R / 2], o[R / 2];
#pragma unroll
        for (int j = 0; j < R / 2; j++) {
            e[j] = v[2 * j];
            o[j] = v[2 * j + 1];
        }
        dft<R / 2, DIR>(e);
        dft<R / 2, DIR>(o);
        dft_combine<R, DIR, 0>(v, e, o);
    }
}

// ----------------------------------------------------- radix plan ----
// A length L = 2^a transform runs as ceil(a/4) Stockham stages whose radices
// (each 2..16) split the a bits as evenly as possible, largest first.
struct RadixPlan {
    int nst;       // number of stages
    int lr[5];     // log2 radix of each stage
};

__host__ __device__ inline RadixPlan make_plan(int log2L)
{
    RadixPlan p;
    p.nst = (log2L + 3) / 4;
    if (p.nst == 0) {
        return p;
    }
    int base = log2L / p.nst, extra = log2L % p.nst;
    for (int s = 0; s < p.nst; s++)
        p.lr[s] = base + (s < extra ? 1 : 0);
    return p;
}

// ------------------------------------------------------------- RK4 ----
// The nonlinear part of Eqs. (CEp)-(CEi) at one point is dA_x/dz = i c_x p_x
// with the products (e = e^{+i dk z})
//   three fields: p_p = A_s A_i e*, p_s = A_p A_i* e, p_i = A_p A_s* e,
//                 c_x = kappa_x;
//   two fields (degenerate): p_p = A_s^2 e*, p_s = A_p A_s* e,
//                 c_p = kappa_p / 2, c_s = kappa_s.
// One classic RK4 step of size h from z0 uses the products at the stage
// points (stage factors e0 = e^{i dk z0}, e1 = e^{i dk (z0 + h/2)},
// e2 = e^{i dk (z0 + h)}); the constants i c_x h/2, i c_x h and i c_x h/6 are
// folded into the fused multiply-adds of the stage updates.  EM: whether the
// phase factors enter (0: never, dk = 0; 2: where the runtime flag use_e says
// so, which compiles to predicated products).
template <int F, int EM, class V>
__device__ __forceinline__ void nl_prod(const V *a, V e, bool use_e, V *p)
{
    if constexpr (F == 3) {
        p[0] = cmul(a[1], a[2]);  // A_s A_i
        p[1] = cmulc(a[0], a[2]); // A_p A_i*
        p[2] = cmulc(a[0], a[1]); // A_p A_s*
        if (EM == 2 && use_e) {
            p[0] = cmulc(p[0], e);
            p[1] = cmul(p[1], e);
            p[2] = cmul(p[2], e);
        }
    } else {
        p[0] = cmul(a[1], a[1]);  // A_s^2
        p[1] = cmulc(a[0], a[1]); // A_p A_s*
        if (EM == 2 && use_e) {
            p[0] = cmulc(p[0], e);
            p[1] = cmul(p[1], e);
        }
    }
}

// y + g (i p) for real g (explicit fused multiply-adds: left to the
// compiler, y - g p may be contracted in one kernel and not in another, and
// two kernels running the same step would not round alike)
template <class V>
__device__ __forceinline__ V add_ig(V y, typename cscal<V>::type g, V p)
{
    return cmk<V>(fmad_(-g, p.y, y.x), fmad_(g, p.x, y.y));
}

// p1 + 2 p2 + 2 p3 + p4, evaluated left to right (the doublings are exact)
template <class V>
__device__ __forceinline__ V rk4_sum(V p1, V p2, V p3, V p4)
{
    using S = typename cscal<V>::type;
    S sx = p1.x + (S)2 * p2.x + (S)2 * p3.x + p4.x;
    S sy = p1.y + (S)2 * p2.y + (S)2 * p3.y + p4.y;
    return cmk<V>(sx, sy);
}

template <int F, int EM, class V>
__device__ __forceinline__ void rk4_point_e(V *y, V e0, V e1, V e2,
                                            const typename cscal<V>::type *kap,
                                            typename cscal<V>::type h, bool use_e)
{
    using S = typename cscal<V>::type;
    S c[F], ch[F], c6[F];
#pragma unroll
    for (int x = 0; x < F; x++) {
        c[x] = (F == 2 && x == 0) ? kap[0] * (S)0.5 : kap[x];
        ch[x] = c[x] * (h * (S)0.5);
        c6[x] = c[x] * (h / (S)6);
        c[x] = c[x] * h;
    }
    V p1[F], p2[F], p3[F], p4[F], t[F];
    nl_prod<F, EM>(y, e0, use_e, p1);
#pragma unroll
    for (int x = 0; x < F; x++)
        t[x] = add_ig(y[x], ch[x], p1[x]);
    nl_prod<F, EM>(t, e1, use_e, p2);
#pragma unroll
    for (int x = 0; x < F; x++)
        t[x] = add_ig(y[x], ch[x], p2[x]);
    nl_prod<F, EM>(t, e1, use_e, p3);
#pragma unroll
    for (int x = 0; x < F; x++)
        t[x] = add_ig(y[x], c[x], p3[x]);
    nl_prod<F, EM>(t, e2, use_e, p4);
#pragma unroll
    for (int x = 0; x < F; x++)
        y[x] = add_ig(y[x], c6[x], rk4_sum(p1[x], p2[x], p3[x], p4[x]));
}

// RK4 step of the same system with the Kerr (chi(3)) terms added:
//   dA_x/dz = i (c_x p_x + g_x A_x),  g_x = sum_y G_xy |A_y|^2,
// where G_xy = (2 pi/lambda_x) n2 n_y eps0 c/2 times 1 (y = x) or 2 (y != x)
// gives self- and cross-phase modulation.  G is row-major 3 x 3.
template <int F, int EM, class V>
__device__ __forceinline__ void rk4_point_kerr_e(V *y, V e0, V e1, V e2,
                                                 const typename cscal<V>::type *kap,
                                                 typename cscal<V>::type h, bool use_e,
                                                 const typename cscal<V>::type *G)
{
    using S = typename cscal<V>::type;
    S c[F];
#pragma unroll
    for (int x = 0; x < F; x++)
        c[x] = (F == 2 && x == 0) ? kap[0] * (S)0.5 : kap[x];
    auto rhs = [&](const V *a, V e, V *q) {
        V p[F];
        nl_prod<F, EM>(a, e, use_e, p);
        S i2[F];
#pragma unroll
        for (int x = 0; x < F; x++)
            i2[x] = cabs2(a[x]);
#pragma unroll
        for (int x = 0; x < F; x++) {
            S g = (S)0;
#pragma unroll
            for (int z = 0; z < F; z++)
                g += G[3 * x + z] * i2[z];
            q[x] = cmk<V>(fmad_(c[x], p[x].x, g * a[x].x), fmad_(c[x], p[x].y, g * a[x].y));
        }
    };
    const S hh = h * (S)0.5, h6 = h / (S)6;
    V q1[F], q2[F], q3[F], q4[F], t[F];
    rhs(y, e0, q1);
#pragma unroll
    for (int x = 0; x < F; x++)
        t[x] = add_ig(y[x], hh, q1[x]);
    rhs(t, e1, q2);
#pragma unroll
    for (int x = 0; x < F; x++)
        t[x] = add_ig(y[x], hh, q2[x]);
    rhs(t, e1, q3);
#pragma unroll
    for (int x = 0; x < F; x++)
        t[x] = add_ig(y[x], h, q3[x]);
    rhs(t, e2, q4);
#pragma unroll
    for (int x = 0; x < F; x++)
        y[x] = add_ig(y[x], h6, rk4_sum(q1[x], q2[x], q3[x], q4[x]));
}

template <int F, class V>
__device__ __forceinline__ void rk4_point(V *y, V e0, V e1, V e2,
                                          const typename cscal<V>::type *kap,
                                          typename cscal<V>::type h, bool use_e)
{
    rk4_point_e<F, 2>(y, e0, e1, e2, kap, h, use_e);
}

template <int F, class V>
__device__ __forceinline__ void rk4_point_kerr(V *y, V e0, V e1, V e2,
                                               const typename cscal<V>::type *kap,
                                               typename cscal<V>::type h, bool use_e,
                                               const typename cscal<V>::type *G)
{
    rk4_point_kerr_e<F, 2>(y, e0, e1, e2, kap, h, use_e, G);
}

// --------------------------------------------------- shared context ----
// Slots of the raw per-round-trip observable sums (FP64): Sum|A_x|^2 for
// x = 0..2, Sum_k |X_k|^2 and Sum_k k'|X_k|^2 of the signal spectrum.
#define OPO_NSLOT 5

// ---------------------------------------------------- Stockham stage ----
// One radix-R stage of a Stockham (autosort, decimation in time) transform
// over nseq sequences of length L held in shared memory.  Butterfly j of a
// sequence reads v_r = src[j + r L/R], multiplies by W_{Ns R}^{DIR r k}
// (k = j mod Ns), takes an R-point DFT and stores output r at position
// (j - k) R + k + r Ns.  After all stages the result is in natural order.
// Element e of sequence seq lives at src[addr(seq, e)]; outputs go through
// store(seq, e, value).  tw[i << twshift] = e^{-2 pi i i'/(Ns R)} ...: the
// table holds W_M^i for a power-of-two M >= Ns R, and twshift = log2(M/(Ns R)).
// SEQ_FAST: consecutive threads take consecutive sequences (column layouts);
// otherwise consecutive butterflies of one sequence (row layouts).
template <int R, int DIR, bool SEQ_FAST, class V, class Addr, class Store>
__device__ __forceinline__ void stockham_stage(const V *__restrict__ src, int nseq, int L, int Ns,
                                               Addr addr, Store store, const V *__restrict__ tw,
                                               int twshift)
{
    const int Lr = L / R;
    const int nbf = nseq * Lr;
    for (int u = threadIdx.x; u < nbf; u += blockDim.x) {
        int seq, j;
        if (SEQ_FAST) {
            seq = u % nseq;
            j = u / nseq;
        } else {
            j = u % Lr;
            seq = u / Lr;
        }
        const int k = j & (Ns - 1);
        V v[R];
#pragma unroll
        for (int r = 0; r < R; r++)
            v[r] = src[addr(seq, j + r * Lr)];
        if (Ns > 1) {
#pragma unroll
            for (int r = 1; r < R; r++) {
                V w = tw[(r * k) << twshift];
                if (DIR > 0)
                    w.y = -w.y;
                v[r] = cmul(v[r], w);
            }
        }
        dft<R, DIR>(v);
        const int base = (j - k) * R + k;
#pragma unroll
        for (int r = 0; r < R; r++)
            store(seq, base + r * Ns, v[r]);
    }
}

// Dispatch a stage by log2 radix.
template <int DIR, bool SEQ_FAST, class V, class Addr, class Store>
__device__ __forceinline__ void stockham_stage_lr(int lr, const V *__restrict__ src, int nseq, int L,
                                                  int Ns, Addr addr, Store store,
                                                  const V *__restrict__ tw, int twshift)
{
    switch (lr) {
    case 1:
        stockham_stage<2, DIR, SEQ_FAST>(src, nseq, L, Ns, addr, store, tw, twshift);
        break;
    case 2:
        stockham_stage<4, DIR, SEQ_FAST>(src, nseq, L, Ns, addr, store, tw, twshift);
        break;
    case 3:
        stockham_stage<8, DIR, SEQ_FAST>(src, nseq, L, Ns, addr, store, tw, twshift);
        break;
    default:
        stockham_stage<16, DIR, SEQ_FAST>(src, nseq, L, Ns, addr, store, tw, twshift);
        break;
    }
}

// Entry pump of the ns-pulsed regime (Sec. 4.2): a Gaussian in intensity,
// much longer than a round trip, read at t = m t_rt + tau_g,
//   A = a0 exp(-c (t - t0)^2),  c = 2 ln 2 / fwhm^2.
// The argument is formed in FP64; the exponential is taken in the field
// precision.
struct NsPump {
    double a0, c, t0, t_rt, dt;
    int n, on;
};

template <class T>
__device__ __forceinline__ cv<T> ns_pump_at(const NsPump &q, int g, int64_t m)
{
    const double t = __fma_rn((double)m, q.t_rt, (double)(g - q.n / 2) * q.dt - q.t0);
    const double x = q.c * t * t;
    T a;
    if constexpr (sizeof(T) == 8)
        a = q.a0 * exp(-x);
    else
        a = (float)q.a0 * expf(-(float)x);
    return cmk<cv<T>>(a, (T)0);
}

__host__ __device__ inline int ilog2(unsigned v)
{
    int r = 0;
    while ((1u << r) < v)
        r++;
    return r;
}
