#pragma once
// opo_fused2.cuh -- fused round-trip kernel specialised at compile time for
// N = P Q with P = 2^LP in {64, 128, 256}, Q = 2^LQ in {64, 128, 256}
// (N = 2^12 ... 2^16; 2^16 in single precision only), field count F and
// precision.  Same method, layout and cluster
// exchange as the generic fused kernel (opo_fused.cu: time domain columns in
// X, frequency-domain rows in Y, two cluster barriers per z-step), with every
// transform split into exactly two Stockham stages whose radices mirror
// between the forward and inverse transform:
//   columns  forward [Ra1, Ra2]   inverse [Ra2, Ra1]
//   rows     forward [Rb1, Rb2]   inverse [Rb2, Rb1]
// so that the inverse column transform's last stage, the two RK4 half steps
// that meet at a z-step boundary (Sec. 2.2: N/2 of step j, then N/2 of step
// j+1) and the next forward column stage all act on the same R values per
// field in one thread's registers ("block A"), and the forward row
// transform's last stage, the dispersion factor and the inverse row
// transform's first stage likewise ("block B").  A z-step is then six
// shared-memory passes:
//   A   S -> X   inverse col stage 2, RK4 x2, forward col stage 1
//   2   X -> Y'  forward col stage 2, W_N^{n2 k1}, push to the owner CTA
//   --- cluster barrier
//   3   Y -> S   forward row stage 1
//   B   S -> Y   forward row stage 2, x D (or G), inverse row stage 1
//   5   Y -> X'  inverse row stage 2, W_N^{-n2 k1}, push to the owner CTA
//   --- cluster barrier
//   6   X -> S   inverse col stage 1
// Rows are stored with an XOR swizzle of the element index so that the
// stride-R stores of a first stage do not collide in shared-memory banks.
#include <cooperative_groups.h>

#include <algorithm>
#include <type_traits>

#include "opo_fused_desc.cuh"

namespace cg = cooperative_groups;

namespace opo {
namespace f2 {

template <class T> struct F2Traits;
template <> struct F2Traits<float> {
    static constexpr int kMaxThreads = 384;
    static constexpr int kSwz = 4; // 16 float2 per 128-byte bank row
};
template <> struct F2Traits<double> {
    static constexpr int kMaxThreads = 256;
    static constexpr int kSwz = 3; // 8 double2 per 128-byte bank row
};

// In-place variant (IP): only the X and Y buffers, so a CTA holds twice the
// points of the S-buffer variant; dispersion factors come from L2.  Every
// in-place stage permutes values within one column or one row, and the work
// items of a column (row) are consecutive threads of one warp, so a warp
// barrier between its reads and its writes is enough.  For that the column
// buffer X is column-major under IP, and both buffers are XOR-swizzled with a
// bit permutation of the column (row) index.
template <class T> struct F2IpTraits;
template <> struct F2IpTraits<float> {
    static constexpr int kMaxThreads = 512; // 16 warps per SM at <= 128 registers
};
template <> struct F2IpTraits<double> {
    static constexpr int kMaxThreads = 256;
};
constexpr int kMaxCl = 16;

template <int R, int DIR, class V>
__device__ __forceinline__ void dft_r(V *v)
{
    dft<R, DIR>(v);
}

// Work items u = threadIdx.x, threadIdx.x + blockDim.x, ... < items of a
// phase that reads one buffer and writes another (the pushes): ld(u, v)
// loads an item's R values, work(u, v) transforms and stores them.  (Issuing
// the next item's loads before the current item's work measured 6% slower.)
template <class V, int R, class Ld, class Work>
__device__ __forceinline__ void items_loop(int items, const Ld &ld, const Work &work)
{
    for (int u = threadIdx.x; u < items; u += blockDim.x) {
        V v[R];
        ld(u, v);
        work(u, v);
    }
}

// Rounds base = 0, blockDim.x, ... < items of an in-place phase: lane
// threadIdx.x takes item base + threadIdx.x (lanes past the end of the last
// round redo item items - 1 and drop it, so that the warp stays converged
// around its barriers); work(u, v, own) transforms and, where own, stores.
template <class V, int R, class Ld, class Work>
__device__ __forceinline__ void rounds_loop(int items, const Ld &ld, const Work &work)
{
#pragma unroll 1
    for (int base = 0; base < items; base += blockDim.x) {
        const int u0 = base + (int)threadIdx.x;
        const int u = u0 < items ? u0 : items - 1;
        V v[R];
        ld(u, v);
        work(u, v, u0 < items);
    }
}

// The W_N^{n2 k1} rotations of the exchange run as a recurrence w <- w step
// along an item's values, taken afresh from the tables every kRotRefresh
// values: each product rounds the modulus, and a recurrence 16 deep left the
// FP32 steady state 1.3e-4 below the oracle's after 20000 round trips (6e-6
// with the refresh, at the same speed).
constexpr int kRotRefresh = 4;
template <class T, bool IP>
constexpr int kF2MaxThreads = IP ? F2IpTraits<T>::kMaxThreads : F2Traits<T>::kMaxThreads;
// Column split [Ra1, Ra2] = [2^A1, 2^A2] of a P = 2^LP column transform:
// A2 = ceil(LP/2), except P = 256, split [8, 32] so that a block-A item keeps
// 8 values per field as at smaller sizes (a [16, 16] split put 16 RK4 points
// of every field in one thread: 255 registers and block A at half speed);
// the 32-point stages go to the column push and the last inverse stage.
constexpr int f2_col_a2(int LP) { return LP == 8 ? 5 : (LP + 1) / 2; }
// Row split [Rb1, Rb2] = [2^B1, 2^B2] of a Q = 2^LQ row transform: B2 =
// ceil(LQ/2), except Q = 512, split [32, 16] so that a block-B item keeps 16
// values (and 16 factors) as at Q = 256; the 32-point stages go to the row
// stage before block B and the inverse push.
constexpr int f2_row_b2(int LQ) { return LQ == 9 ? 4 : (LQ + 1) / 2; }

// P = 256 (N = 2^16, 2^17): the 32-point column stages need more than 128
// registers: at most 384 threads in FP32, 256 in FP64 (up to 255 registers).
// P = 128 (N = 2^14, 2^15), three FP32 fields in place, chi(2): at most 256
// threads, so that up to 255 registers are available; the fastest shape for
// a batch (8-CTA clusters of 128 threads, two CTAs per SM) ran 2.4% faster
// than under the 128-register cap of 512 threads (1.907 against 1.954 ms,
// bit-identical results).  Two fields and the Kerr variant keep 512-thread
// CTAs.
template <class T, int F, bool IP, int LP, int NL>
constexpr int kF2MaxThreadsL =
    LP >= 8 ? (sizeof(T) == 8 ? 256 : 384)
            : ((IP && sizeof(T) == 4 && F == 3 && LP == 7 && NL != kNlKerr)
                   ? 256
                   : kF2MaxThreads<T, IP>);

// NL: the nonlinear-step variant (kNlChi2, kNlKerr, kNlChi2NoDk), each a
// separate instantiation so that every kernel carries only the arithmetic
// (and the registers) its instances need.
//
// XG (with IP): the exchange between CTAs goes through two global buffers of
// the instance (F N values each, L2-resident) instead of the owners' shared
// memory, and X and Y are one buffer: a CTA holds only N/C points per field
// once, so three FP32 fields at N = 2^17, or FP64 at 2^16, fit a 16-CTA
// cluster.  The forward push writes G1 in the natural row-major order of the
// frequency rows, [f][k1][n2]; after the cluster barrier each CTA's first row
// stage reads its rows from G1 into Y (X's space: every CTA has read its own
// columns before the barrier).  The inverse push writes G2 in the time-domain
// order [f][n1][n2]; after the second barrier the first inverse column stage
// reads its columns from G2 into X.  Each buffer is written only between the
// barrier that follows its last reads and the barrier that precedes its next
// reads, so the two cluster barriers per z-step still suffice.
template <class T, int F, int LP, int LQ, bool IP, int NL, bool XG = false, int CC = 0>
__global__ void __launch_bounds__(kF2MaxThreadsL<T, F, IP, LP, NL>, 1)
    k_fused2(const InstDesc *__restrict__ descs, int r_base, int M, int write_out, int disp_smem)
{
    static_assert(!XG || IP, "the exchange through global memory uses the in-place layouts");
    constexpr bool KR = NL == kNlKerr;
    using V = cv<T>;
    constexpr int P = 1 << LP, Q = 1 << LQ, LN = LP + LQ, N = 1 << LN;
    constexpr int A2 = f2_col_a2(LP), A1 = LP - A2; // columns [Ra1, Ra2]
    constexpr int B2 = f2_row_b2(LQ), B1 = LQ - B2; // rows    [Rb1, Rb2]
    constexpr int Ra1 = 1 << A1, Ra2 = 1 << A2, Rb1 = 1 << B1, Rb2 = 1 << B2;
    constexpr int LS = (LN + 1) / 2; // W_N^a = hi[a >> LS] lo[a & (2^LS - 1)]
    constexpr int SW = F2Traits<T>::kSwz;
    constexpr int SWM = (1 << SW) - 1;

    cg::cluster_group cluster = cg::this_cluster();
    const int C = CC ? CC : (int)cluster.num_blocks(); // CC: the cluster size, if compiled in
    const int c = (int)cluster.block_rank();
    const int inst = blockIdx.x / C;
    const int logC = ilog2((unsigned)C);
    const int logPc = LP - logC, logQc = LQ - logC;
    const int Pc = 1 << logPc, Qc = 1 << logQc;
    const int NC = N >> logC;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    V *X = reinterpret_cast<V *>(smem_raw);
    V *Y = XG ? X : X + F * NC;
    V *S = IP ? nullptr : Y + F * NC;
    V *Dsm = IP ? Y + F * NC : S + F * NC;
    // stage twiddles W^{r j}, indexed [r][j] with j the butterfly index that
    // runs along consecutive lanes: the loads of one r hit consecutive
    // words (or one broadcast word) and sit at constant offsets from the
    // item's base
    V *twA = Dsm + (disp_smem ? F * NC : 0); // W_P, r < Ra1, j < Ra2 (block A)
    V *tw2 = twA + P;                         // W_P, r < Ra2, j < Ra1 (phase 2)
    V *twB = tw2 + P;                         // W_Q, r < Rb2, j < Rb1 (block B)
    V *tw5 = twB + Q;                         // W_Q, r < Rb1, j < Rb2 (phase 5)
    V *twLo = tw5 + Q;
    V *twHi = twLo + (1 << LS);
    double *red = reinterpret_cast<double *>(twHi + (N >> LS));
    __shared__ V *rX[kMaxCl];
    __shared__ V *rY[kMaxCl];

    // ---- descriptor scalars into registers
    const InstDesc &dg = descs[inst];
    const unsigned resmask = dg.resmask;
    const int ncry = dg.ncry;
    const bool eom = dg.eom != 0;
    constexpr bool kerr = KR;
    // constants of every crystal of the round trip, in the field precision
    struct CrySm {
        T kap[3], h;
        T G[KR ? 9 : 1]; // Kerr coefficients G_xy
        const V *ekz;    // e^{i dk q dz/4}
        const V *D;      // dispersion factors: row-major (IP) or natural order
        int nz, use_e;
    };
    __shared__ CrySm sCry[kMaxCry];
    if (threadIdx.x < ncry) {
        const CryDesc &cd = dg.cry[threadIdx.x];
        CrySm &s = sCry[threadIdx.x];
        for (int x = 0; x < 3; x++)
            s.kap[x] = (T)cd.kappa[x];
        s.h = (T)cd.h;
        if constexpr (KR)
            for (int i = 0; i < 9; i++)
                s.G[i] = (T)cd.kerr_g[i];
        s.ekz = (const V *)cd.ekz;
        s.D = (const V *)(IP ? cd.disp_t : cd.disp);
        s.nz = cd.nz;
        s.use_e = cd.use_dk;
    }
    V bc[3], osc[3];
    for (int x = 0; x < 3; x++) {
        bc[x] = cmk<V>((T)dg.bc_re[x], (T)dg.bc_im[x]);
        osc[x] = cmk<V>((T)dg.outscale[x], (T)0);
    }
    const double eom_beta = dg.eom_beta, eom_f = dg.eom_f, t_rt = dg.t_rt, dt = dg.dt;
    const int64_t m_start = dg.m_start;
    V *gF = (V *)dg.fields;
    V *gOut = (V *)dg.out;
    V *gHist = (V *)dg.hist;
    const V *gPump = (const V *)dg.pump;
    const V *gD = (const V *)dg.disp;
    const V *gG = (const V *)dg.gdd;
    const V *gGt = (const V *)dg.gdd_t;
    const V *gtw = (const V *)dg.tw;
    double *obs = dg.obs;
    int *err = dg.err;
    V *G1 = (V *)dg.xg1; // XG: forward exchange, [f][k1][n2]
    V *G2 = (V *)dg.xg2; // XG: inverse exchange, [f][n1][n2]
    (void)G1;
    (void)G2;

    // W_P^e = gtw[e << LQ], W_Q^e = gtw[e << LP]
    for (int i = threadIdx.x; i < P; i += blockDim.x) {
        twA[i] = gtw[((i >> A2) * (i & (Ra2 - 1))) << LQ];
        tw2[i] = gtw[((i >> A1) * (i & (Ra1 - 1))) << LQ];
    }
    for (int i = threadIdx.x; i < Q; i += blockDim.x) {
        twB[i] = gtw[((i >> B1) * (i & (Rb1 - 1))) << LP];
        tw5[i] = gtw[((i >> B2) * (i & (Rb2 - 1))) << LP];
    }
    for (int i = threadIdx.x; i < (1 << LS); i += blockDim.x)
        twLo[i] = gtw[i];
    for (int i = threadIdx.x; i < (N >> LS); i += blockDim.x)
        twHi[i] = gtw[i << LS];
    if (threadIdx.x < C) {
        rX[threadIdx.x] = cluster.map_shared_rank(X, (unsigned)threadIdx.x);
        rY[threadIdx.x] = cluster.map_shared_rank(Y, (unsigned)threadIdx.x);
    }
    if (disp_smem) {
        for (int i = threadIdx.x; i < F * NC; i += blockDim.x) {
            int f = i / NC, p = i - f * NC;
            int row = p >> LQ, k2 = p & (Q - 1);
            Dsm[i] = gD[f * N + (c << logPc) + row + (k2 << LP)];
        }
    }

    // ---- index helpers
    auto cidx = [=](int f, int n1, int b) { return f * NC + (n1 << logQc) + b; };
    // rows: the element index is XOR-swizzled within 2^SW-element groups by
    // its group number and by the row, so that both unit-stride and stride-R
    // accesses of one or two rows per wavefront hit distinct banks
    auto ridx = [=](int f, int row, int e) {
        return f * NC + (row << LQ) + (e ^ (((e >> SW) ^ (row << (SW - 1))) & SWM));
    };
    // IP layouts: perm(x) puts neighbours x, x+1 in different halves of a
    // 2^SW-element bank group and maps 2^SW aligned consecutive x to distinct
    // values, so column (row) and cross-column (cross-row) accesses both avoid
    // bank conflicts
    auto perm = [](int x) {
        return (((x & 1) << (SW - 1)) | ((x >> 1) & ((1 << (SW - 1)) - 1))) & SWM;
    };
    auto cidx_ip = [=](int f, int n1, int b) {
        return f * NC + (b << LP) + (n1 ^ (((n1 >> SW) ^ perm(b)) & SWM));
    };
    auto ridx_ip = [=](int f, int row, int e) {
        return f * NC + (row << LQ) + (e ^ (((e >> SW) ^ perm(row)) & SWM));
    };
    auto CI = [=](int f, int n1, int b) { return IP ? cidx_ip(f, n1, b) : cidx(f, n1, b); };
    auto RI = [=](int f, int row, int e) { return IP ? ridx_ip(f, row, e) : ridx(f, row, e); };
    // IP accesses of one work item touch the elements e0 | x of one column
    // (row), x = r R a compile-time constant with bits disjoint from e0.  The
    // swizzle is linear over the bits of the element index, so that element
    // sits at the byte offset (a0 ^ lo(x)) + hi(x) from the first one's
    // offset a0: one logic operation per access, the rest an immediate.
    // (Buffer and column/row starts are multiples of 128 bytes, so the XOR
    // stays within the swizzled bits.)
    auto ipo = [&](const V *buf, int i0) -> unsigned {
        return (unsigned)((const unsigned char *)(buf + i0) - smem_raw);
    };
    auto ipx = [&](unsigned a0, int x) -> V & {
        const unsigned lo = (unsigned)(((x ^ (x >> SW)) & SWM) * (int)sizeof(V));
        const unsigned hi = (unsigned)((x & ~SWM) * (int)sizeof(V));
        return *reinterpret_cast<V *>(smem_raw + ((a0 ^ lo) + hi));
    };
    auto gtime = [=](int n1, int b) { return (n1 << LQ) + (c << logQc) + b; };
    auto twN = [&](unsigned a) {
        a &= (unsigned)(N - 1);
        return cmul(twHi[a >> LS], twLo[a & ((1u << LS) - 1)]);
    };

    // ---- IP pushes: for the unrolled position r of a phase-2 (phase-5) item,
    // the address in the owner CTA of the start of the destination row
    // (column) group and the swizzle term of that group's row (column)
    // number; the item's own part of the destination index is XORed with the
    // latter and added to the former (row and swizzle are both linear in the
    // bits of the row (column) index).  Holds when a CTA owns at least one
    // butterfly group along the destination direction (Pc >= Ra1,
    // Qc >= Rb2).  Taken for clusters of one or two CTAs (+5% at 2^12, +2.5%
    // at 2^13); with more destinations the per-element table loads cost more
    // than the index arithmetic they replace (-1 to -3% at 2^14..2^16), and
    // the pushes compute the index per element.
    struct __align__(16) PushEnt {
        unsigned char *p;
        unsigned x;
    };
    __shared__ PushEnt sPush2[IP ? Ra2 : 1], sPush5[IP ? Rb1 : 1];
    const bool tab2 = IP && C <= 2 && Pc >= Ra1, tab5 = IP && C <= 2 && Qc >= Rb2;
    if constexpr (IP) {
        if (tab2 && (int)threadIdx.x < Ra2) {
            const int k1 = (int)threadIdx.x * Ra1, R = k1 & (Pc - 1);
            V *dY = cluster.map_shared_rank(Y, (unsigned)(k1 >> logPc));
            sPush2[threadIdx.x].p = (unsigned char *)(dY + (R << LQ));
            sPush2[threadIdx.x].x = (unsigned)(sizeof(V) * perm(R));
        }
        if (tab5 && (int)threadIdx.x < Rb1) {
            const int n2 = (int)threadIdx.x * Rb2, B = n2 & (Qc - 1);
            V *dX = cluster.map_shared_rank(X, (unsigned)(n2 >> logQc));
            sPush5[threadIdx.x].p = (unsigned char *)(dX + (B << LP));
            sPush5[threadIdx.x].x = (unsigned)(sizeof(V) * perm(B));
        }
    }

    // ---- constants of the crystal being passed (registers, as for one
    // crystal); set_crystal switches them where the next crystal begins
    T kap[3], h;
    bool use_e;
    const V *ekz;
    int kcur;
    auto set_crystal = [&](int k) {
        kcur = k;
        for (int x = 0; x < 3; x++)
            kap[x] = sCry[k].kap[x];
        h = sCry[k].h;
        use_e = sCry[k].use_e != 0;
        ekz = sCry[k].ekz;
    };

    // ---- one RK4 half step (Sec. 2.2) at each of a block-A item's Ra1 points:
    // without any phase-factor products in the dk = 0 variant, else with them
    // predicated on the crystal's flag
    auto rk4_item = [&](V (&v)[F][Ra1], V e0, V e1, V e2) {
        constexpr int EM = NL == kNlChi2NoDk ? 0 : 2;
#pragma unroll
        for (int r = 0; r < Ra1; r++) {
            V y[F];
#pragma unroll
            for (int f = 0; f < F; f++)
                y[f] = v[f][r];
            if constexpr (kerr)
                rk4_point_kerr_e<F, EM>(y, e0, e1, e2, kap, h, use_e, sCry[kcur].G);
            else
                rk4_point_e<F, EM>(y, e0, e1, e2, kap, h, use_e);
#pragma unroll
            for (int f = 0; f < F; f++)
                v[f][r] = y[f];
        }
    };

    // ---- block A: shared by every z-step boundary
    // mode 0: first round trip of the launch, input from global memory
    // mode 1: interior z-step boundary
    // mode 2: end of the crystal pass (observables and outputs, with the
    //         output history row m_cav, then cavity forward)
    // mode 3: end of the cavity visit of round trip m_cav (mirror, EOM, then
    //         entry of round trip m_cav + 1, or the final store)
    // modes 5 and 6: a z-step boundary where one crystal ends and the next
    //         begins, in two passes with the current crystal's constants
    //         each: 5 ends the step (inverse column stage 2, RK4 half step)
    //         and stores the time-domain values where it read them, 6 takes
    //         them up again (RK4 half step of the next crystal, forward
    //         column stage 1); each item stays with the same thread
    auto block_a = [&](auto mode_tag, int qa, int qb, int64_t m_cav, bool next_rt, bool save_out,
                       double *acc) {
        constexpr int mode = decltype(mode_tag)::value;
        const V e0a = use_e ? ekz[qa] : cmk<V>((T)1, (T)0);
        const V e1a = use_e ? ekz[qa + 1] : e0a;
        const V e2a = use_e ? ekz[qa + 2] : e0a;
        const V e0b = use_e ? ekz[qb] : cmk<V>((T)1, (T)0);
        const V e1b = use_e ? ekz[qb + 1] : e0b;
        const V e2b = use_e ? ekz[qb + 2] : e0b;
        // work item u -> (column b, butterfly j < Ra2); IP keeps a column's
        // items in consecutive threads
        auto dec = [&](int u, int &b, int &j) {
            if constexpr (IP) {
                j = u & (Ra2 - 1);
                b = u >> A2;
            } else {
                b = u & (Qc - 1);
                j = u >> logQc;
            }
        };
        auto load = [&](int u, V (&v)[F][Ra1]) {
            int b, j;
            dec(u, b, j);
            if constexpr (mode == 0) {
#pragma unroll
                for (int r = 0; r < Ra1; r++) {
                    const int g = gtime(j + r * Ra2, b);
#pragma unroll
                    for (int f = 0; f < F; f++)
                        v[f][r] = gF[f * N + g];
                }
            } else {
                const V *src = IP ? X : S;
                (void)src;
#pragma unroll
                for (int f = 0; f < F; f++) {
                    if constexpr (IP) {
                        const unsigned a0 = ipo(X, CI(f, j, b));
#pragma unroll
                        for (int r = 0; r < Ra1; r++)
                            v[f][r] = ipx(a0, r * Ra2);
                    } else {
#pragma unroll
                        for (int r = 0; r < Ra1; r++)
                            v[f][r] = src[CI(f, j + r * Ra2, b)];
                    }
                }
            }
        };
        // own: this lane owns work item u (lanes past the end of the last
        // round redo an item only to keep the warp converged; their
        // observables must not count)
        auto process = [&](int u, V (&v)[F][Ra1], bool own) -> bool {
            int b, j;
            dec(u, b, j);
            if constexpr (mode != 0 && mode != 6) {
                // inverse column stage 2: radix Ra1, Ns = Ra2, k = j
#pragma unroll
                for (int f = 0; f < F; f++) {
#pragma unroll
                    for (int r = 1; r < Ra1; r++) {
                        V w = twA[r * Ra2 + j];
                        w.y = -w.y;
                        v[f][r] = cmul(v[f][r], w);
                    }
                    dft_r<Ra1, 1>(v[f]);
                }
            }
            // time domain: v[f][r] at n1 = j + r Ra2
            if constexpr (mode == 1 || mode == 2 || mode == 5)
                rk4_item(v, e0a, e1a, e2a);
            if constexpr (mode == 2) {
#pragma unroll
                for (int r = 0; r < Ra1; r++) {
#pragma unroll
                    for (int f = 0; f < F; f++) {
                        if (own)
                            acc[f] += (double)cabs2(v[f][r]);
                        if (save_out && own)
                            gOut[f * N + gtime(j + r * Ra2, b)] = cmul(v[f][r], osc[f]);
                        // output history: row m_cav (the round trip's slot in
                        // the call) in mode 2
                        if (gHist && own)
                            gHist[(size_t)m_cav * F * N + f * N + gtime(j + r * Ra2, b)] =
                                cmul(v[f][r], osc[f]);
                    }
                }
            }
            if constexpr (mode == 3) {
#pragma unroll
                for (int r = 0; r < Ra1; r++) {
                    V mod = cmk<V>((T)1, (T)0);
                    if (eom) {
                        const int gi = gtime(j + r * Ra2, b);
                        double uu = __fma_rn(eom_f, (double)(gi - N / 2) * dt,
                                             eom_f * ((double)m_cav * t_rt));
                        double fr = uu - floor(uu);
                        T ph;
                        if constexpr (sizeof(T) == 8)
                            ph = (T)(eom_beta * sinpi(2.0 * fr));
                        else
                            ph = (T)eom_beta * sinpif((T)2 * (T)fr);
                        T sn, cs;
                        sincos(ph, &sn, &cs);
                        mod = cmk<V>(cs, sn);
                    }
#pragma unroll
                    for (int f = 0; f < F; f++) {
                        if (resmask & (1u << f)) {
                            V t = cmul(v[f][r], bc[f]);
                            v[f][r] = eom ? cmul(t, mod) : t;
                        }
                    }
                }
                if (!next_rt) {
                    if (own) {
#pragma unroll
                        for (int r = 0; r < Ra1; r++)
#pragma unroll
                            for (int f = 0; f < F; f++)
                                gF[f * N + gtime(j + r * Ra2, b)] = v[f][r];
                    }
                    return false;
                }
            }
            if constexpr (mode == 0 || mode == 3) {
                // entry of a round trip, then its first RK4 half step
#pragma unroll
                for (int r = 0; r < Ra1; r++) {
                    // the input pump replaces a non-resonant pump and is added
                    // to a resonant one; non-resonant s/i restart from zero
                    const int g = gtime(j + r * Ra2, b);
                    const V pin = dg.ns.on ? ns_pump_at<T>(dg.ns, g, m_cav + 1) : gPump[g];
                    v[0][r] = (resmask & 1u) ? cadd(v[0][r], pin) : pin;
#pragma unroll
                    for (int f = 1; f < F; f++)
                        if (!(resmask & (1u << f)))
                            v[f][r] = cmk<V>((T)0, (T)0);
                }
                rk4_item(v, e0b, e1b, e2b);
            } else if constexpr (mode == 1 || mode == 6) {
                rk4_item(v, e0b, e1b, e2b);
            }
            // forward column stage 1: radix Ra1, Ns = 1, outputs at j Ra1 + r
            if constexpr (mode != 5) {
#pragma unroll
                for (int f = 0; f < F; f++)
                    dft_r<Ra1, -1>(v[f]);
            }
            return true;
        };
        auto store = [&](int u, V (&v)[F][Ra1]) {
            int b, j;
            dec(u, b, j);
            if constexpr (mode == 5) {
                // time domain, back where the values came from
                V *dst = IP ? X : S;
                (void)dst;
#pragma unroll
                for (int f = 0; f < F; f++) {
                    if constexpr (IP) {
                        const unsigned a0 = ipo(X, CI(f, j, b));
#pragma unroll
                        for (int r = 0; r < Ra1; r++)
                            ipx(a0, r * Ra2) = v[f][r];
                    } else {
#pragma unroll
                        for (int r = 0; r < Ra1; r++)
                            dst[CI(f, j + r * Ra2, b)] = v[f][r];
                    }
                }
            } else {
#pragma unroll
                for (int f = 0; f < F; f++) {
                    if constexpr (IP) {
                        const unsigned a0 = ipo(X, CI(f, j * Ra1, b));
#pragma unroll
                        for (int r = 0; r < Ra1; r++)
                            ipx(a0, r) = v[f][r];
                    } else {
#pragma unroll
                        for (int r = 0; r < Ra1; r++)
                            X[CI(f, j * Ra1 + r, b)] = v[f][r];
                    }
                }
            }
        };
        if constexpr (IP && mode != 0) {
            // in place on X: a column's reads and writes stay within one warp
            const int items = Qc << A2;
#pragma unroll 1
            for (int base = 0; base < items; base += blockDim.x) {
                // lanes past the end redo the last item and drop it, so the
                // warp stays converged around the barrier (warps wholly past
                // the end run the round too: letting them skip it measured
                // 1-8% slower)
                const int u0 = base + threadIdx.x;
                const bool have = u0 < items;
                const int u = have ? u0 : items - 1;
                V v[F][Ra1];
                load(u, v);
                const bool st = process(u, v, have) && have;
                __syncwarp();
                if (st)
                    store(u, v);
                __syncwarp();
            }
        } else {
            for (int u = threadIdx.x; u < (Qc << A2); u += blockDim.x) {
                V v[F][Ra1];
                load(u, v);
                if (process(u, v, true))
                    store(u, v);
            }
        }
    };

    // ---- phase 2: forward column stage 2 and push into the owners' Y
    // Consecutive lanes take consecutive columns b: each remote store of a
    // warp then writes whole 128-byte runs of one destination row (the
    // swizzles keep the column reads free of bank conflicts under IP too).
    auto phase2 = [&]() {
        const int items = F * Qc * Ra1;
        auto ld = [&](int u, V (&v)[Ra2]) {
            const int b = u & (Qc - 1);
            const int rest = u >> logQc;
            const int j = rest & (Ra1 - 1), f = rest >> A1;
            if constexpr (IP) {
                const unsigned a0 = ipo(X, CI(f, j, b));
#pragma unroll
                for (int r = 0; r < Ra2; r++)
                    v[r] = ipx(a0, r * Ra1);
            } else {
#pragma unroll
                for (int r = 0; r < Ra2; r++)
                    v[r] = X[CI(f, j + r * Ra1, b)];
            }
        };
        auto work = [&](int u, V (&v)[Ra2]) {
            const int b = u & (Qc - 1);
            const int rest = u >> logQc;
            const int j = rest & (Ra1 - 1), f = rest >> A1;
#pragma unroll
            for (int r = 1; r < Ra2; r++)
                v[r] = cmul(v[r], tw2[r * Ra1 + j]);
            dft_r<Ra2, -1>(v);
            const int n2 = (c << logQc) + b;
            // W_N^{n2 k1} for k1 = j + r Ra1: base W_N^{n2 j} times step^r
            const V step = twN((unsigned)(n2 * Ra1));
            V w = twN((unsigned)(n2 * j));
            if constexpr (XG) {
                // row k1 = j + r Ra1 of G1, column n2: consecutive lanes write
                // consecutive n2
                V *g = G1 + (size_t)f * N + (size_t)j * Q + n2;
#pragma unroll
                for (int r = 0; r < Ra2; r++) {
                    if (r > 0 && r % kRotRefresh == 0)
                        w = twN((unsigned)(n2 * (j + r * Ra1)));
                    __stcg(g + (size_t)r * Ra1 * Q, cmul(v[r], w));
                    w = cmul(w, step);
                }
            } else if (tab2) {
                const unsigned a0 = (unsigned)(sizeof(V) * RI(f, j, n2));
#pragma unroll
                for (int r = 0; r < Ra2; r++) {
                    const PushEnt t = sPush2[r];
                    if (r > 0 && r % kRotRefresh == 0)
                        w = twN((unsigned)(n2 * (j + r * Ra1)));
                    *reinterpret_cast<V *>(t.p + (a0 ^ t.x)) = cmul(v[r], w);
                    w = cmul(w, step);
                }
            } else {
#pragma unroll
                for (int r = 0; r < Ra2; r++) {
                    const int k1 = j + r * Ra1;
                    if (r > 0 && r % kRotRefresh == 0)
                        w = twN((unsigned)(n2 * k1));
                    rY[k1 >> logPc][RI(f, k1 & (Pc - 1), n2)] = cmul(v[r], w);
                    w = cmul(w, step);
                }
            }
        };
        items_loop<V, Ra2>(items, ld, work);
    };

    // ---- phase 3: forward row stage 1, Y -> S (in place on Y for IP)
    auto phase3 = [&]() {
        const int items = F * Pc * Rb2;
        auto dec = [&](int u, int &j, int &row, int &f) {
            j = u & (Rb2 - 1);
            const int rest = u >> B2;
            row = rest & (Pc - 1);
            f = rest >> logPc;
        };
        if constexpr (XG) {
            // the CTA's rows from G1 (consecutive lanes read consecutive
            // elements of a row), written to Y: no in-place hazard
            for (int u = threadIdx.x; u < items; u += blockDim.x) {
                int j, row, f;
                dec(u, j, row, f);
                const V *src = G1 + (size_t)f * N + (size_t)((c << logPc) + row) * Q + j;
                V v[Rb1];
#pragma unroll
                for (int r = 0; r < Rb1; r++)
                    v[r] = __ldcg(src + r * Rb2);
                dft_r<Rb1, -1>(v);
                const unsigned a1 = ipo(Y, RI(f, row, j * Rb1));
#pragma unroll
                for (int r = 0; r < Rb1; r++)
                    ipx(a1, r) = v[r];
            }
        } else if constexpr (IP) {
            auto ld = [&](int u, V (&v)[Rb1]) {
                int j, row, f;
                dec(u, j, row, f);
                const unsigned a0 = ipo(Y, RI(f, row, j));
#pragma unroll
                for (int r = 0; r < Rb1; r++)
                    v[r] = ipx(a0, r * Rb2);
            };
            auto work = [&](int u, V (&v)[Rb1], bool have) {
                int j, row, f;
                dec(u, j, row, f);
                dft_r<Rb1, -1>(v);
                __syncwarp();
                if (have) {
                    const unsigned a1 = ipo(Y, RI(f, row, j * Rb1));
#pragma unroll
                    for (int r = 0; r < Rb1; r++)
                        ipx(a1, r) = v[r];
                }
                __syncwarp();
            };
            rounds_loop<V, Rb1>(items, ld, work);
        } else {
            for (int u = threadIdx.x; u < items; u += blockDim.x) {
                int j, row, f;
                dec(u, j, row, f);
                V v[Rb1];
#pragma unroll
                for (int r = 0; r < Rb1; r++)
                    v[r] = Y[ridx(f, row, j + r * Rb2)];
                dft_r<Rb1, -1>(v);
#pragma unroll
                for (int r = 0; r < Rb1; r++)
                    S[ridx(f, row, j * Rb1 + r)] = v[r];
            }
        }
    };

    // ---- block B: forward row stage 2, spectral factor, inverse row stage 1
    // cav (compile time): the cavity visit (GDD/delay factor, spectrum sums)
    // instead of a z-step's dispersion factor
    auto block_b = [&](auto cav_tag, double *acc, int kc) {
        constexpr bool cav = decltype(cav_tag)::value;
        const int items = F * Pc * Rb1;
        const V *Dk = sCry[kc].D; // dispersion factors of crystal kc
        const bool dsm = disp_smem && kc == 0;
        const V *src = IP ? Y : S;
        (void)dsm;
        (void)src;
        auto decode = [&](int u, int &j, int &row, int &f) {
            j = u & (Rb1 - 1);
            const int rest = u >> B1;
            row = rest & (Pc - 1);
            f = rest >> logPc;
        };
        auto load = [&](int u, V (&v)[Rb2]) {
            int j, row, f;
            decode(u, j, row, f);
            if constexpr (IP) {
                const unsigned a0 = ipo(Y, RI(f, row, j));
#pragma unroll
                for (int r = 0; r < Rb2; r++)
                    v[r] = ipx(a0, r * Rb1);
            } else {
#pragma unroll
                for (int r = 0; r < Rb2; r++)
                    v[r] = src[RI(f, row, j + r * Rb1)];
            }
        };
        auto finish = [&](int u, V (&v)[Rb2], bool own) {
            int j, row, f;
            decode(u, j, row, f);
            const int k1 = (c << logPc) + row;
            // IP: the factors come from L2, from the row-major copy, so that
            // a warp's loads (consecutive j) coalesce; issued before the
            // transform so that their latency overlaps it
            V fac[IP ? Rb2 : 1];
            (void)fac;
            if constexpr (IP) {
                const V *tab = (cav ? gGt : Dk) + f * N + (k1 << LQ) + j;
#pragma unroll
                for (int r = 0; r < Rb2; r++)
                    fac[r] = tab[r * Rb1];
            }
#pragma unroll
            for (int r = 1; r < Rb2; r++)
                v[r] = cmul(v[r], twB[r * Rb1 + j]);
            dft_r<Rb2, -1>(v);
#pragma unroll
            for (int r = 0; r < Rb2; r++) {
                const int k2 = j + r * Rb1;
                const int k = k1 + (k2 << LP);
                V d;
                if constexpr (IP)
                    d = fac[r];
                else
                    d = cav ? gG[f * N + k] : (dsm ? Dsm[f * NC + (row << LQ) + k2] : Dk[f * N + k]);
                if (cav && f == 1 && own) {
                    double p2 = (double)cabs2(v[r]);
                    acc[3] += p2;
                    acc[4] = __fma_rn((double)((k < N / 2) ? k : k - N), p2, acc[4]);
                }
                v[r] = cmul(v[r], d);
            }
            dft_r<Rb2, 1>(v);
        };
        auto store = [&](int u, V (&v)[Rb2]) {
            int j, row, f;
            decode(u, j, row, f);
            if constexpr (IP) {
                const unsigned a0 = ipo(Y, RI(f, row, j * Rb2));
#pragma unroll
                for (int r = 0; r < Rb2; r++)
                    ipx(a0, r) = v[r];
            } else {
#pragma unroll
                for (int r = 0; r < Rb2; r++)
                    Y[RI(f, row, j * Rb2 + r)] = v[r];
            }
        };
        if constexpr (IP) {
            auto work = [&](int u, V (&v)[Rb2], bool have) {
                finish(u, v, have);
                __syncwarp();
                if (have)
                    store(u, v);
                __syncwarp();
            };
            rounds_loop<V, Rb2>(items, load, work);
        } else {
            for (int u = threadIdx.x; u < items; u += blockDim.x) {
                V v[Rb2];
                load(u, v);
                finish(u, v, true);
                store(u, v);
            }
        }
    };

    // ---- phase 5: inverse row stage 2 and push into the owners' X
    // The destination X is row-major without IP (consecutive lanes take
    // consecutive butterflies j, i.e. consecutive columns n2) and column-major
    // with IP (consecutive lanes take consecutive rows k1); either way a warp's
    // remote store writes whole 128-byte runs.
    auto phase5 = [&]() {
        const int items = F * Pc * Rb2;
        auto dec5 = [&](int u, int &j, int &row, int &f) {
            if constexpr (IP && !XG) {
                row = u & (Pc - 1);
                const int rest = u >> logPc;
                j = rest & (Rb2 - 1);
                f = rest >> B2;
            } else {
                j = u & (Rb2 - 1);
                const int rest = u >> B2;
                row = rest & (Pc - 1);
                f = rest >> logPc;
            }
        };
        auto ld = [&](int u, V (&v)[Rb1]) {
            int j, row, f;
            dec5(u, j, row, f);
            if constexpr (IP) {
                const unsigned a0 = ipo(Y, RI(f, row, j));
#pragma unroll
                for (int r = 0; r < Rb1; r++)
                    v[r] = ipx(a0, r * Rb2);
            } else {
#pragma unroll
                for (int r = 0; r < Rb1; r++)
                    v[r] = Y[RI(f, row, j + r * Rb2)];
            }
        };
        auto work = [&](int u, V (&v)[Rb1]) {
            int j, row, f;
            dec5(u, j, row, f);
#pragma unroll
            for (int r = 1; r < Rb1; r++) {
                V w = tw5[r * Rb2 + j];
                w.y = -w.y;
                v[r] = cmul(v[r], w);
            }
            dft_r<Rb1, 1>(v);
            const int k1 = (c << logPc) + row;
            // W_N^{-n2 k1} for n2 = j + r Rb2: base W_N^{-k1 j} times step^r
            V step = twN((unsigned)(k1 * Rb2));
            step.y = -step.y;
            V w = twN((unsigned)(k1 * j));
            w.y = -w.y;
            if constexpr (XG) {
                // row n1 = k1 of G2, columns n2 = j + r Rb2: consecutive lanes
                // write consecutive n2
                V *g = G2 + (size_t)f * N + (size_t)k1 * Q + j;
#pragma unroll
                for (int r = 0; r < Rb1; r++) {
                    if (r > 0 && r % kRotRefresh == 0) {
                        w = twN((unsigned)(k1 * (j + r * Rb2)));
                        w.y = -w.y;
                    }
                    __stcg(g + r * Rb2, cmul(v[r], w));
                    w = cmul(w, step);
                }
            } else if (tab5) {
                const unsigned a0 = (unsigned)(sizeof(V) * CI(f, k1, j));
#pragma unroll
                for (int r = 0; r < Rb1; r++) {
                    const PushEnt t = sPush5[r];
                    if (r > 0 && r % kRotRefresh == 0) {
                        w = twN((unsigned)(k1 * (j + r * Rb2)));
                        w.y = -w.y;
                    }
                    *reinterpret_cast<V *>(t.p + (a0 ^ t.x)) = cmul(v[r], w);
                    w = cmul(w, step);
                }
            } else {
#pragma unroll
                for (int r = 0; r < Rb1; r++) {
                    const int n2 = j + r * Rb2;
                    if (r > 0 && r % kRotRefresh == 0) {
                        w = twN((unsigned)(k1 * n2));
                        w.y = -w.y;
                    }
                    rX[n2 >> logQc][CI(f, k1, n2 & (Qc - 1))] = cmul(v[r], w);
                    w = cmul(w, step);
                }
            }
        };
        items_loop<V, Rb1>(items, ld, work);
    };

    // ---- phase 6: inverse column stage 1, X -> S (in place on X for IP)
    auto phase6 = [&]() {
        const int items = F * Qc * Ra1;
        if constexpr (XG) {
            // the CTA's columns from G2 (consecutive lanes read consecutive
            // columns of a row), written to X: no in-place hazard
            for (int u = threadIdx.x; u < items; u += blockDim.x) {
                const int b = u & (Qc - 1);
                const int rest = u >> logQc;
                const int j = rest & (Ra1 - 1), f = rest >> A1;
                const V *src = G2 + (size_t)f * N + (size_t)j * Q + (c << logQc) + b;
                V v[Ra2];
#pragma unroll
                for (int r = 0; r < Ra2; r++)
                    v[r] = __ldcg(src + (size_t)r * Ra1 * Q);
                dft_r<Ra2, 1>(v);
                const unsigned a1 = ipo(X, cidx_ip(f, j * Ra2, b));
#pragma unroll
                for (int r = 0; r < Ra2; r++)
                    ipx(a1, r) = v[r];
            }
        } else if constexpr (IP) {
            auto dec6 = [&](int u, int &j, int &b, int &f) {
                j = u & (Ra1 - 1);
                const int rest = u >> A1;
                b = rest & (Qc - 1);
                f = rest >> logQc;
            };
            auto ld = [&](int u, V (&v)[Ra2]) {
                int j, b, f;
                dec6(u, j, b, f);
                const unsigned a0 = ipo(X, cidx_ip(f, j, b));
#pragma unroll
                for (int r = 0; r < Ra2; r++)
                    v[r] = ipx(a0, r * Ra1);
            };
            auto work = [&](int u, V (&v)[Ra2], bool have) {
                int j, b, f;
                dec6(u, j, b, f);
                dft_r<Ra2, 1>(v);
                __syncwarp();
                if (have) {
                    const unsigned a1 = ipo(X, cidx_ip(f, j * Ra2, b));
#pragma unroll
                    for (int r = 0; r < Ra2; r++)
                        ipx(a1, r) = v[r];
                }
                __syncwarp();
            };
            rounds_loop<V, Ra2>(items, ld, work);
        } else {
            for (int u = threadIdx.x; u < items; u += blockDim.x) {
                const int b = u & (Qc - 1);
                const int rest = u >> logQc;
                const int j = rest & (Ra1 - 1), f = rest >> A1;
                V v[Ra2];
#pragma unroll
                for (int r = 0; r < Ra2; r++)
                    v[r] = X[cidx(f, j + r * Ra1, b)];
                dft_r<Ra2, 1>(v);
#pragma unroll
                for (int r = 0; r < Ra2; r++)
                    S[cidx(f, j * Ra2 + r, b)] = v[r];
            }
        }
    };

    // forward transform (after block A), frequency visit, inverse up to S
    // XG: the pushes went to global memory; a device-scope fence before the
    // cluster barrier makes them visible to the other CTAs (which read them
    // past L1)
    auto xsync = [&]() {
        if constexpr (XG)
            __threadfence();
        cluster.sync();
    };
    auto middle = [&](auto cav_tag, double *acc, int kc) {
        __syncthreads();
        phase2();
        xsync();
        phase3();
        __syncthreads();
        block_b(cav_tag, acc, kc);
        __syncthreads();
        phase5();
        xsync();
        phase6();
        __syncthreads();
    };

    using M0 = std::integral_constant<int, 0>;
    using M1 = std::integral_constant<int, 1>;
    using M2 = std::integral_constant<int, 2>;
    using M3 = std::integral_constant<int, 3>;
    using M5 = std::integral_constant<int, 5>;
    using M6 = std::integral_constant<int, 6>;
    cluster.sync(); // every CTA of the cluster is running; tables loaded
    double dummy[kNslot] = {0, 0, 0, 0, 0};
    // mode 0 enters round trip m_start + r_base (its m_cav is the one before)
    set_crystal(0);
    block_a(M0{}, 0, 0, m_start + r_base - 1, true, false, dummy);
    for (int r = 0; r < M; r++) {
        const int64_t slot = (int64_t)r_base + r;
        const int64_t m = m_start + slot;
        // the z-steps of every crystal in order (step jz of crystal kc); at a
        // boundary between two steps block A finishes one and starts the
        // next, possibly in the next crystal (z restarts there: its stage
        // factors from q = 0).  Few live registers: the crystal's step count
        // is re-read from shared memory.
        int jz = 0;
        while (kcur + 1 < ncry || jz + 1 < sCry[kcur].nz) {
            middle(std::false_type{}, dummy, kcur);
            if (jz + 1 < sCry[kcur].nz) {
                block_a(M1{}, 4 * jz + 2, 4 * (jz + 1), 0, true, false, dummy);
                jz++;
            } else {
                block_a(M5{}, 4 * jz + 2, 0, 0, true, false, dummy);
                set_crystal(kcur + 1);
                __syncthreads();
                block_a(M6{}, 0, 0, 0, true, false, dummy);
                jz = 0;
            }
        }
        middle(std::false_type{}, dummy, kcur);
        double acc[kNslot] = {0, 0, 0, 0, 0};
        block_a(M2{}, 4 * jz + 2, 0, slot, true, write_out && r == M - 1, acc);
        middle(std::true_type{}, acc, 0);
        block_reduce5(acc, red);
        if (threadIdx.x == 0) {
            double *o = obs + (slot * C + c) * kNslot;
            for (int q = 0; q < kNslot; q++)
                o[q] = acc[q];
            if (!isfinite(acc[0] + acc[1] + acc[2]))
                atomicOr(err, 1);
        }
        set_crystal(0);
        block_a(M3{}, 0, 0, m, r + 1 < M, false, dummy);
    }
}

template <class T, int F, int LP, int LQ, bool IP, int NL, bool XG, int CC = 0>
int launch_t(const InstDesc *dd, int count, int C, int threads, size_t sm, bool disp_smem,
             int r_base, int chunk, int last, cudaStream_t s)
{
    auto kern = k_fused2<T, F, LP, LQ, IP, NL, XG, CC>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3(count * C);
    lc.blockDim = dim3(threads);
    lc.dynamicSmemBytes = sm;
    lc.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    lc.attrs = at;
    lc.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&lc, kern, dd, r_base, chunk, last, (int)disp_smem);
    return e == cudaSuccess ? OPO_OK : OPO_E_CUDA;
}

template <class T, int F, int LP, int LQ, bool IP, int NL, bool XG, int CC = 0>
int max_active_t(int C, int threads, size_t sm)
{
    auto kern = k_fused2<T, F, LP, LQ, IP, NL, XG, CC>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3(C);
    lc.blockDim = dim3(threads);
    lc.dynamicSmemBytes = sm;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    lc.attrs = at;
    lc.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, kern, &lc) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nclusters;
}

// Launch (op 0) or occupancy query (op 1) of every instantiated size for one
// precision and field count; ip selects the in-place variant, nl the
// nonlinear-step variant.  The variants of a precision and field count are
// defined in separate translation units (opo_fused2_<prec>_<F>.cu, ..._kerr.cu
// and, single precision only, ..._nodk.cu) that compile in parallel.
#define OPO_F2_DISPATCH_DECL(NAME)                                                               \
    int NAME(int op, bool ip, int nl, int logn, const InstDesc *dd, int count, int C,            \
             int threads, size_t sm, bool ds, int r_base, int chunk, int last, cudaStream_t s)
#define OPO_F2_DISPATCH_NL_DECL(NAME)                                                            \
    int NAME(int op, bool ip, int logn, const InstDesc *dd, int count, int C, int threads,       \
             size_t sm, bool ds, int r_base, int chunk, int last, cudaStream_t s)
OPO_F2_DISPATCH_DECL(dispatch_f32_f3);
OPO_F2_DISPATCH_DECL(dispatch_f32_f2);
OPO_F2_DISPATCH_DECL(dispatch_f64_f3);
OPO_F2_DISPATCH_DECL(dispatch_f64_f2);
OPO_F2_DISPATCH_NL_DECL(dispatch_f32_f3_kerr);
OPO_F2_DISPATCH_NL_DECL(dispatch_f32_f2_kerr);
OPO_F2_DISPATCH_NL_DECL(dispatch_f64_f3_kerr);
OPO_F2_DISPATCH_NL_DECL(dispatch_f64_f2_kerr);
OPO_F2_DISPATCH_NL_DECL(dispatch_f32_f3_nodk);
OPO_F2_DISPATCH_NL_DECL(dispatch_f32_f2_nodk);

// Launch (op 0) or occupancy query (op 1) of one instantiation.
// The cluster size compiled into an instantiation's batch shape, or 0 (a
// runtime value): three FP32 fields, chi(2), in place: 8-CTA clusters at
// 2^14, 16-CTA clusters at 2^16.  Exchange indices and cluster arithmetic
// then become constants, with bit-identical results: 1.837 against 1.910 ms
// per round trip of 36 instances at 2^14, 1.478 against 1.560 ms for 7
// sync-pumped instances at 2^16.  (The FP64 2^14 kernel, bound by the FP64
// pipe, gained nothing: 30.87 against 30.85 ms.)
template <class T, int F, int LP, int LQ, bool IP, int NL, bool XG>
constexpr int f2_compiled_cluster()
{
    if (!IP || XG || F != 3 || NL == kNlKerr || sizeof(T) != 4)
        return 0;
    if (LP == 7 && LQ == 7)
        return 8;
    if (LP == 8 && LQ == 8)
        return 16;
    return 0;
}

template <class T, int F, int LP, int LQ, bool IP, int NL, bool XG>
int one_t(int op, const InstDesc *dd, int count, int C, int threads, size_t sm, bool ds,
          int r_base, int chunk, int last, cudaStream_t s)
{
    constexpr int CC = f2_compiled_cluster<T, F, LP, LQ, IP, NL, XG>();
    if constexpr (CC > 0) {
        if (C == CC)
            return op == 0 ? launch_t<T, F, LP, LQ, IP, NL, XG, CC>(dd, count, C, threads, sm, ds,
                                                                    r_base, chunk, last, s)
                           : max_active_t<T, F, LP, LQ, IP, NL, XG, CC>(C, threads, sm);
    }
    return op == 0 ? launch_t<T, F, LP, LQ, IP, NL, XG>(dd, count, C, threads, sm, ds, r_base,
                                                        chunk, last, s)
                   : max_active_t<T, F, LP, LQ, IP, NL, XG>(C, threads, sm);
}

// Every size for one (T, F, NL).  A function template, so that the branches
// `if constexpr` discards (sizes a precision does not have) are not compiled.
// In place: 2^12..2^16 exchange through the owners' shared memory; three
// FP32 fields at 2^17 and FP64 at 2^16 exchange through global memory.
template <class T, int F, int NL>
int sizes_t(int op, bool ip, int logn, const InstDesc *dd, int count, int C, int threads,
            size_t sm, bool ds, int r_base, int chunk, int last, cudaStream_t s)
{
    constexpr bool F32 = sizeof(T) == 4;
    const int none = op == 0 ? OPO_E_UNSUPPORTED : 0;
#define OPO_F2_ONE(LP, LQ, IP, XG)                                                               \
    return one_t<T, F, LP, LQ, IP, NL, XG>(op, dd, count, C, threads, sm, ds, r_base, chunk,     \
                                           last, s)
    if (ip) {
        switch (logn) {
        case 12:
            OPO_F2_ONE(6, 6, true, false);
        case 13:
            OPO_F2_ONE(6, 7, true, false);
        case 14:
            OPO_F2_ONE(7, 7, true, false);
        case 15:
            OPO_F2_ONE(7, 8, true, false);
        case 16:
            if constexpr (F32) {
                OPO_F2_ONE(8, 8, true, false);
            } else {
                OPO_F2_ONE(8, 8, true, true);
            }
        case 17:
            if constexpr (F32) {
                OPO_F2_ONE(8, 9, true, true);
            } else {
                return none;
            }
        default:
            return none;
        }
    }
    switch (logn) {
    case 12:
        OPO_F2_ONE(6, 6, false, false);
    case 13:
        OPO_F2_ONE(6, 7, false, false);
    case 14:
        OPO_F2_ONE(7, 7, false, false);
    case 15:
        OPO_F2_ONE(7, 8, false, false);
    case 16:
        if constexpr (F32) {
            OPO_F2_ONE(8, 8, false, false);
        } else {
            return none;
        }
    default:
        return none;
    }
#undef OPO_F2_ONE
}

#define OPO_F2_SIZES(T, F, NL)                                                                   \
    return sizes_t<T, F, NL>(op, ip, logn, dd, count, C, threads, sm, ds, r_base, chunk, last, s);

// the general chi(2) sizes, and the entry point that forwards the other
// variants to their translation units (FP64 has no dk = 0 variant)
#define OPO_F2_DISPATCH_DEF(NAME, T, F)                                                          \
    OPO_F2_DISPATCH_DECL(NAME)                                                                   \
    {                                                                                            \
        if (nl == kNlKerr)                                                                       \
            return NAME##_kerr(op, ip, logn, dd, count, C, threads, sm, ds, r_base, chunk,       \
                               last, s);                                                         \
        OPO_F2_SIZES(T, F, kNlChi2)                                                              \
    }

#define OPO_F2_DISPATCH_DEF_NODK(NAME, T, F)                                                     \
    OPO_F2_DISPATCH_DECL(NAME)                                                                   \
    {                                                                                            \
        if (nl == kNlKerr)                                                                       \
            return NAME##_kerr(op, ip, logn, dd, count, C, threads, sm, ds, r_base, chunk,       \
                               last, s);                                                         \
        if (nl == kNlChi2NoDk)                                                                   \
            return NAME##_nodk(op, ip, logn, dd, count, C, threads, sm, ds, r_base, chunk,       \
                               last, s);                                                         \
        OPO_F2_SIZES(T, F, kNlChi2)                                                              \
    }

#define OPO_F2_DISPATCH_KERR_DEF(NAME, T, F)                                                     \
    OPO_F2_DISPATCH_NL_DECL(NAME##_kerr)                                                         \
    {                                                                                            \
        OPO_F2_SIZES(T, F, kNlKerr)                                                              \
    }

#define OPO_F2_DISPATCH_NODK_DEF(NAME, T, F)                                                     \
    OPO_F2_DISPATCH_NL_DECL(NAME##_nodk)                                                         \
    {                                                                                            \
        OPO_F2_SIZES(T, F, kNlChi2NoDk)                                                          \
    }

} // namespace f2
} // namespace opo
