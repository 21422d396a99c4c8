// opo_fused.cu -- the fused form of the OPO round trip (arXiv 2410.02532,
// Sec. 2.2 split-step with RK4, Sec. 2.1 Eq. (BC), Sec. 2.3, main loop of
// Sec. 4.1): one persistent kernel in which a thread-block cluster of C CTAs
// holds all fields of one instance in distributed shared memory for many
// round trips.  HBM is read at launch start (fields, tables) and written at
// launch end (fields, output fields, observable partial sums).
//
// Data layout.  N = P Q, time index n = Q n1 + n2, frequency index
// k = k1 + P k2 (n1, k1 < P; n2, k2 < Q); Pc = P/C, Qc = Q/C.
//   time domain (buffer X of CTA c): x[n1][n2] for n2 in [c Qc, c Qc + Qc),
//     stored at f*NC + n1*Qc + (n2 - c Qc)
//   frequency domain (buffer Y of CTA c): X[k1][k2] for k1 in
//     [c Pc, c Pc + Pc), stored at f*NC + (k1 - c Pc)*Q + k2
// with NC = N/C points per field per CTA.
//
// One forward FFT: P-point column transforms of X (local), twiddle
// W_N^{n2 k1}, store straight into the owner CTA's Y over DSMEM, cluster
// barrier, Q-point row transforms of Y (local).  The inverse runs the same
// path backwards.  RK4 and the pointwise cavity elements act on X, the
// dispersion and GDD factors on Y, so each z-step costs exactly two cluster
// barriers and two all-to-all exchanges.
//
// Buffer discipline (why two barriers per z-step suffice): a CTA pushes into
// remote Y only between the inverse barrier of the previous step and the
// forward barrier of this one, when no CTA reads its own Y; it pushes into
// remote X only between the forward and inverse barriers, when no CTA reads
// its own X.  S is private scratch for the ping-pong of Stockham stages.
#include <algorithm>
#include <cstddef>
#include <type_traits>
#include <vector>

#include <cooperative_groups.h>

#include "opo_fused_desc.cuh"

namespace cg = cooperative_groups;

namespace opo {
namespace {

constexpr int kMaxCluster = 16;
constexpr int kFusedThreads = 256;

template <class T>
__global__ void __launch_bounds__(kFusedThreads, 1)
    k_fused(const InstDesc *__restrict__ descs, int r_base, int M, int write_out, int disp_smem,
            int fmax, int nc_max, int lmax_max)
{
    using V = cv<T>;
    cg::cluster_group cluster = cg::this_cluster();
    const int C = (int)cluster.num_blocks();
    const int c = (int)cluster.block_rank();
    const int inst = blockIdx.x / C;
    const InstDesc &d = descs[inst];

    const int n = d.n, logn = d.logn, F = d.F;
    const int logP = d.logP, logQ = d.logQ;
    const int P = 1 << logP, Q = 1 << logQ;
    const int logC = ilog2((unsigned)C);
    const int logPc = logP - logC, logQc = logQ - logC;
    const int Pc = 1 << logPc, Qc = 1 << logQc;
    const int NC = n >> logC;
    const int logL = logP > logQ ? logP : logQ; // twiddle table of the sub-transforms
    const int logS = (logn + 1) / 2;            // split of W_N^a = hi[a >> logS] lo[a & mask]

    // ---- shared memory carve-up (sized for the largest instance) ----
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V *X = reinterpret_cast<V *>(smem_raw);
    V *Y = X + (size_t)fmax * nc_max;
    V *S = Y + (size_t)fmax * nc_max;
    V *Dsm = S + (size_t)fmax * nc_max;
    V *twL = Dsm + (disp_smem ? (size_t)fmax * nc_max : 0);
    V *twLo = twL + lmax_max;
    V *twHi = twLo + (1 << ((17 + 1) / 2));
    double *red = reinterpret_cast<double *>(twHi + (1 << (17 / 2)));
    __shared__ V *rX[kMaxCluster];
    __shared__ V *rY[kMaxCluster];

    const V *gtw = (const V *)d.tw;
    for (int i = threadIdx.x; i < (1 << logL); i += blockDim.x)
        twL[i] = gtw[(size_t)i << (logn - logL)];
    for (int i = threadIdx.x; i < (1 << logS); i += blockDim.x)
        twLo[i] = gtw[i];
    for (int i = threadIdx.x; i < (n >> logS); i += blockDim.x)
        twHi[i] = gtw[(size_t)i << logS];
    if (threadIdx.x < C) {
        rX[threadIdx.x] = cluster.map_shared_rank(X, (unsigned)threadIdx.x);
        rY[threadIdx.x] = cluster.map_shared_rank(Y, (unsigned)threadIdx.x);
    }
    // state and dispersion slice
    V *gF = (V *)d.fields;
    for (int i = threadIdx.x; i < F * NC; i += blockDim.x) {
        int f = i / NC, p = i - f * NC;
        int n1 = p >> logQc, n2l = p & (Qc - 1);
        X[i] = gF[(size_t)f * n + ((size_t)n1 << logQ) + (c << logQc) + n2l];
    }
    const V *gD = (const V *)d.disp;
    if (disp_smem) {
        for (int i = threadIdx.x; i < F * NC; i += blockDim.x) {
            int f = i / NC, p = i - f * NC;
            int k1l = p >> logQ, k2 = p & (Q - 1);
            Dsm[i] = gD[(size_t)f * n + (c << logPc) + k1l + ((size_t)k2 << logP)];
        }
    }
    // constants of the crystal being passed (several per round trip)
    T kap[3], h, kg[9];
    bool use_e = false, kerr = false;
    const V *ekz = nullptr;
    const V *gDk = gD;
    int nzk = 0;
    auto load_crystal = [&](int k) {
        const CryDesc &cd = d.cry[k];
        for (int x = 0; x < 3; x++)
            kap[x] = (T)cd.kappa[x];
        h = (T)cd.h;
        use_e = cd.use_dk != 0;
        kerr = cd.kerr != 0;
        for (int i = 0; i < 9; i++)
            kg[i] = (T)cd.kerr_g[i];
        ekz = (const V *)cd.ekz;
        gDk = (const V *)cd.disp;
        nzk = cd.nz;
    };
    const V *gG = (const V *)d.gdd;
    const V *gPump = (const V *)d.pump;
    const RadixPlan planP = make_plan(logP), planQ = make_plan(logQ);
    cluster.sync(); // every CTA of the cluster is running and loaded

    // W_N^{a}, a taken mod N
    auto twN = [&](unsigned a) -> V {
        a &= (unsigned)(n - 1);
        return cmul(twHi[a >> logS], twLo[a & ((1u << logS) - 1)]);
    };
    auto addrA = [=](int seq, int e) { // column seq = f*Qc + b, element n1 = e
        int f = seq >> logQc, b = seq & (Qc - 1);
        return f * NC + (e << logQc) + b;
    };
    auto addrC = [=](int seq, int e) { return (seq << logQ) + e; }; // row seq = f*Pc + k1l

    // Run the stages of a sub-transform except the last one, ping-ponging
    // between `home` and S; returns the buffer that holds the last stage's
    // input.  Stage twiddles come from twL (size 2^logL).
    auto stages_but_last = [&](auto dir_tag, bool cols, V *home, const RadixPlan &pl, int L,
                               int nseq, int &Ns) -> V * {
        constexpr int DIR = decltype(dir_tag)::value;
        V *src = home;
        for (int s = 0; s + 1 < pl.nst; s++) {
            const int lr = pl.lr[s];
            V *dst = (src == S) ? home : S;
            const int tsh = logL - (ilog2((unsigned)Ns) + lr);
            if (cols) {
                auto st = [dst, addrA](int seq, int e, V v) { dst[addrA(seq, e)] = v; };
                stockham_stage_lr<DIR, true>(lr, src, nseq, L, Ns, addrA, st, twL, tsh);
            } else {
                auto st = [dst, addrC](int seq, int e, V v) { dst[addrC(seq, e)] = v; };
                stockham_stage_lr<DIR, false>(lr, src, nseq, L, Ns, addrC, st, twL, tsh);
            }
            __syncthreads();
            src = dst;
            Ns <<= lr;
        }
        return src;
    };

    using FWD = std::integral_constant<int, -1>;
    using INV = std::integral_constant<int, 1>;

    // forward transform of every field: X (time) -> Y (frequency, remote)
    auto forward_to_Y = [&]() {
        int Ns = 1;
        V *src = stages_but_last(FWD{}, true, X, planP, P, F * Qc, Ns);
        const int lr = planP.lr[planP.nst - 1];
        const int tsh = logL - (ilog2((unsigned)Ns) + lr);
        auto st = [&](int seq, int k1, V v) {
            int f = seq >> logQc, b = seq & (Qc - 1);
            int n2 = (c << logQc) + b;
            V w = twN((unsigned)n2 * (unsigned)k1);
            int dst = k1 >> logPc, k1l = k1 & (Pc - 1);
            rY[dst][f * NC + (k1l << logQ) + n2] = cmul(v, w);
        };
        stockham_stage_lr<-1, true>(lr, src, F * Qc, P, Ns, addrA, st, twL, tsh);
        cluster.sync();
    };

    // row transforms of Y, multiply by a spectral factor, inverse row
    // transforms, push back into remote X, inverse column transforms.
    // Returns the buffer holding the time-domain result.  `spec` accumulates
    // the signal spectrum sums (cavity visit).
    auto freq_visit_and_back = [&](bool use_gdd, double *acc, bool dsm) -> V * {
        // forward rows
        int Ns = 1;
        V *src = stages_but_last(FWD{}, false, Y, planQ, Q, F * Pc, Ns);
        int lr = planQ.lr[planQ.nst - 1];
        int tsh = logL - (ilog2((unsigned)Ns) + lr);
        V *dstb = (src == S) ? Y : S;
        auto st_mul = [&](int seq, int k2, V v) {
            int f = seq >> logPc, k1l = seq & (Pc - 1);
            int k = (c << logPc) + k1l + (k2 << logP);
            V fac;
            if (use_gdd) {
                fac = gG[(size_t)f * n + k];
                if (f == 1) {
                    double p2 = (double)cabs2(v);
                    int kk = (k < (n >> 1)) ? k : k - n;
                    acc[3] += p2;
                    acc[4] = __fma_rn((double)kk, p2, acc[4]);
                }
            } else {
                fac = dsm ? Dsm[(seq << logQ) + k2] : gDk[(size_t)f * n + k];
            }
            dstb[addrC(seq, k2)] = cmul(v, fac);
        };
        stockham_stage_lr<-1, false>(lr, src, F * Pc, Q, Ns, addrC, st_mul, twL, tsh);
        __syncthreads();
        // inverse rows, home buffer is wherever the data now lives
        Ns = 1;
        V *home = dstb;
        src = home;
        for (int s = 0; s + 1 < planQ.nst; s++) {
            const int lr2 = planQ.lr[s];
            V *dst = (src == S) ? Y : S;
            const int t2 = logL - (ilog2((unsigned)Ns) + lr2);
            auto st = [dst, addrC](int seq, int e, V v) { dst[addrC(seq, e)] = v; };
            stockham_stage_lr<1, false>(lr2, src, F * Pc, Q, Ns, addrC, st, twL, t2);
            __syncthreads();
            src = dst;
            Ns <<= lr2;
        }
        lr = planQ.lr[planQ.nst - 1];
        tsh = logL - (ilog2((unsigned)Ns) + lr);
        auto st_back = [&](int seq, int n2, V v) {
            int f = seq >> logPc, k1l = seq & (Pc - 1);
            int k1 = (c << logPc) + k1l;
            V w = twN((unsigned)n2 * (unsigned)k1);
            w.y = -w.y;
            int dst = n2 >> logQc, n2l = n2 & (Qc - 1);
            rX[dst][f * NC + (k1 << logQc) + n2l] = cmul(v, w);
        };
        stockham_stage_lr<1, false>(lr, src, F * Pc, Q, Ns, addrC, st_back, twL, tsh);
        cluster.sync();
        // inverse columns: all stages regular, result in X or S
        Ns = 1;
        src = X;
        for (int s = 0; s < planP.nst; s++) {
            const int lr2 = planP.lr[s];
            V *dst = (src == S) ? X : S;
            const int t2 = logL - (ilog2((unsigned)Ns) + lr2);
            auto st = [dst, addrA](int seq, int e, V v) { dst[addrA(seq, e)] = v; };
            stockham_stage_lr<1, true>(lr2, src, F * Qc, P, Ns, addrA, st, twL, t2);
            __syncthreads();
            src = dst;
            Ns <<= lr2;
        }
        return src;
    };

    // RK4 half step on every point of the CTA: reads `src`, writes X.
    auto rk4_half = [&](const V *src, int q0) {
        const V e0 = ekz[q0], e1 = ekz[q0 + 1], e2 = ekz[q0 + 2];
        for (int p = threadIdx.x; p < NC; p += blockDim.x) {
            V y[3];
            y[2] = cmk<V>((T)0, (T)0);
            for (int f = 0; f < F; f++)
                y[f] = src[f * NC + p];
            if (kerr) {
                if (F == 3)
                    rk4_point_kerr<3>(y, e0, e1, e2, kap, h, use_e, kg);
                else
                    rk4_point_kerr<2>(y, e0, e1, e2, kap, h, use_e, kg);
            } else if (F == 3) {
                rk4_point<3>(y, e0, e1, e2, kap, h, use_e);
            } else {
                rk4_point<2>(y, e0, e1, e2, kap, h, use_e);
            }
            for (int f = 0; f < F; f++)
                X[f * NC + p] = y[f];
        }
    };

    auto gindex = [=](int p) -> int { // global time index of local position p
        int n1 = p >> logQc, n2l = p & (Qc - 1);
        return (n1 << logQ) + (c << logQc) + n2l;
    };

    for (int r = 0; r < M; r++) {
        const int64_t slot = (int64_t)r_base + r;
        const int64_t m = d.m_start + slot;
        // ---- entry: the input pump replaces a non-resonant pump and is added
        // to a resonant one; non-resonant s/i restart from zero
        for (int i = threadIdx.x; i < F * NC; i += blockDim.x) {
            const int f = i / NC;
            const bool res = (d.resmask >> f) & 1u;
            if (f == 0) {
                const int g = gindex(i);
                const V pin = d.ns.on ? ns_pump_at<T>(d.ns, g, m) : gPump[g];
                X[i] = res ? cadd(X[i], pin) : pin;
            } else if (!res) {
                X[i] = cmk<V>((T)0, (T)0);
            }
        }
        __syncthreads();
        // ---- crystal passes: nz symmetrized steps of every crystal in order
        for (int kc = 0; kc < d.ncry; kc++) {
            load_crystal(kc);
            for (int j = 0; j < nzk; j++) {
                rk4_half(X, 4 * j);
                __syncthreads();
                forward_to_Y();
                V *res = freq_visit_and_back(false, nullptr, disp_smem && kc == 0);
                rk4_half(res, 4 * j + 2);
                __syncthreads();
            }
        }
        // ---- observables: output power sums, non-finite check
        double acc[kNslot] = {0, 0, 0, 0, 0};
        for (int i = threadIdx.x; i < F * NC; i += blockDim.x) {
            int f = i / NC;
            acc[f] += (double)cabs2(X[i]);
        }
        if (d.hist) { // output history row of this round trip
            V *row = (V *)d.hist + (size_t)slot * F * n;
            for (int i = threadIdx.x; i < F * NC; i += blockDim.x) {
                int f = i / NC;
                row[(size_t)f * n + gindex(i - f * NC)] = cscale(X[i], (T)d.outscale[f]);
            }
        }
        if (write_out && r == M - 1) {
            V *go = (V *)d.out;
            for (int i = threadIdx.x; i < F * NC; i += blockDim.x) {
                int f = i / NC;
                go[(size_t)f * n + gindex(i - f * NC)] = cscale(X[i], (T)d.outscale[f]);
            }
        }
        __syncthreads();
        // ---- cavity: spectral visit (GDD, delay, signal spectrum sums)
        forward_to_Y();
        V *res = freq_visit_and_back(true, acc, false);
        block_reduce5(acc, red);
        if (threadIdx.x == 0) {
            double *o = d.obs + (slot * C + c) * kNslot;
            for (int q = 0; q < kNslot; q++)
                o[q] = acc[q];
            if (!isfinite(acc[0] + acc[1] + acc[2]))
                atomicOr(d.err, 1);
        }
        // ---- mirror sqrt(R) e^{i delta}, then EOM, on resonant fields
        for (int p = threadIdx.x; p < NC; p += blockDim.x) {
            V mod = cmk<V>((T)1, (T)0);
            if (d.eom) {
                int gi = gindex(p);
                double u = d.eom_f * ((double)(gi - n / 2) * d.dt) + d.eom_f * ((double)m * d.t_rt);
                double fr = u - floor(u);
                T ph;
                if constexpr (sizeof(T) == 8)
                    ph = (T)(d.eom_beta * sinpi(2.0 * fr));
                else
                    ph = (T)d.eom_beta * sinpif((T)2 * (T)fr);
                T sn, cs;
                sincos(ph, &sn, &cs);
                mod = cmk<V>(cs, sn);
            }
            for (int f = 0; f < F; f++) {
                V v = res[f * NC + p];
                if (d.resmask & (1u << f)) {
                    v = cmul(v, cmk<V>((T)d.bc_re[f], (T)d.bc_im[f]));
                    if (d.eom)
                        v = cmul(v, mod);
                }
                X[f * NC + p] = v;
            }
        }
        __syncthreads();
    }
    // ---- write the state back
    for (int i = threadIdx.x; i < F * NC; i += blockDim.x) {
        int f = i / NC;
        gF[(size_t)f * n + gindex(i - f * NC)] = X[i];
    }
}

size_t smem_bytes(size_t csz, int fmax, int nc_max, int lmax, bool disp_smem)
{
    size_t el = (size_t)fmax * nc_max * (disp_smem ? 4 : 3) + lmax + (1 << 9) + (1 << 8);
    return el * csz + 32 * kNslot * sizeof(double);
}

constexpr size_t kSmemLimit = 227 * 1024;
constexpr int kTargetNc = 2048;
// N <= 2^13: the size-specialised kernels start from 4096 points per field in
// each CTA (one CTA at 2^12, two at 2^13, in place), 14-22% more throughput
// than 2048 (and no cluster exchange at all at 2^12); larger sizes keep 2048,
// which halves a lone instance's round-trip time for a few percent of batch
// throughput (the autotuner picks per class)
constexpr int kTargetNc2Small = 4096;

template <class T>
int max_active(int C, size_t sm)
{
    cudaFuncSetAttribute(k_fused<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    cudaFuncSetAttribute(k_fused<T>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3(C);
    lc.blockDim = dim3(kFusedThreads);
    lc.dynamicSmemBytes = sm;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    lc.attrs = at;
    lc.numAttrs = 1;
    int nclusters = 0;
    cudaError_t e = cudaOccupancyMaxActiveClusters(&nclusters, k_fused<T>, &lc);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nclusters;
}

bool cluster_launchable(bool dbl, int C, size_t sm)
{
    return (dbl ? max_active<double>(C, sm) : max_active<float>(C, sm)) > 0;
}

} // namespace

bool fused_config(size_t csz, int fmin, int fmax, int nmin, int nmax, int cluster_req,
                  int rtpl_req, int threads_req, int nl, FusedCfg *out)
{
    const bool dbl = csz == sizeof(double2);
    const int lognmin = ilog2((unsigned)nmin), lognmax = ilog2((unsigned)nmax);
    // one size and one field count: the size-specialised kernel if it holds it
    if (nmin == nmax && fmin == fmax) {
        // default: about kTargetNc points per field in each CTA (the shape the
        // headline size runs best in), then larger, then smaller clusters
        int c0 = nmax <= 8192 ? nmax / kTargetNc2Small : nmax / kTargetNc;
        c0 = c0 < 1 ? 1 : (c0 > 16 ? 16 : c0);
        int order[5], no = 0;
        for (int c = c0; c <= 16; c *= 2)
            order[no++] = c;
        for (int c = c0 / 2; c >= 1; c /= 2)
            order[no++] = c;
        for (int i = 0; i < no; i++) {
            if (cluster_req > 0 && order[i] != cluster_req)
                continue;
            if (fused2_config(dbl, nl, fmax, lognmax, order[i], threads_req, out)) {
                out->rt_per_launch = rtpl_req > 0 ? rtpl_req : 64;
                return true;
            }
        }
    }
    if (threads_req > 0 && threads_req != kFusedThreads)
        return false; // the generic kernel runs kFusedThreads threads
    const int logPmin = lognmin / 2;
    const int lmax = 1 << (lognmax - lognmax / 2); // Q >= P, so the largest sub-length is Q
    // Default: the smallest cluster that keeps at most kTargetNc points per
    // field in each CTA (more CTAs than that buy little against the
    // exchange); otherwise the largest cluster that fits.
    const int cands[5] = {1, 2, 4, 8, 16};
    FusedCfg best{};
    bool found = false;
    for (int i = 0; i < 5; i++) {
        const int C = cands[i];
        if (cluster_req > 0 && C != cluster_req)
            continue;
        if ((1 << logPmin) < C)
            continue; // every CTA owns at least one row of every instance
        const int nc = nmax / C;
        for (int ds = 1; ds >= 0; ds--) {
            const size_t sm = smem_bytes(csz, fmax, nc, lmax, ds == 1);
            if (sm > kSmemLimit)
                continue;
            if (!cluster_launchable(dbl, C, sm))
                break;
            best.kernel = 1;
            best.nl = nl; // the generic kernel branches on the flags at run time
            best.cluster = C;
            best.threads = kFusedThreads;
            best.rt_per_launch = rtpl_req > 0 ? rtpl_req : 64;
            best.disp_in_smem = ds == 1;
            best.smem = sm;
            found = true;
            break;
        }
        if (found && (cluster_req > 0 || nc <= kTargetNc))
            break;
    }
    if (found)
        *out = best;
    return found;
}

int fused_max_active(bool dbl, int F, int n, const FusedCfg &cfg)
{
    if (cfg.kernel >= 2)
        return fused2_max_active(dbl, F, ilog2((unsigned)n), cfg);
    return dbl ? max_active<double>(cfg.cluster, cfg.smem) : max_active<float>(cfg.cluster, cfg.smem);
}

void fill_desc(InstDesc &d, const opo_ctx *c)
{
    d.fields = c->d_fields;
    d.out = c->d_out;
    d.hist = c->d_hist;
    d.pump = c->d_pump;
    d.disp = c->d_disp;
    d.gdd = c->d_gdd;
    d.disp_t = c->d_disp_t;
    d.gdd_t = c->d_gdd_t;
    d.tw = c->d_tw;
    d.ekz = c->d_ekz;
    d.obs = c->d_obs;
    d.trace = c->d_trace;
    d.err = (int *)((char *)c->d_ctl + offsetof(DevCtl, err));
    d.n = c->n;
    d.logn = c->logn;
    d.logP = c->logn / 2;
    d.logQ = c->logn - d.logP;
    d.F = c->F;
    d.nz = c->crystal.nz;
    d.resmask = c->cavity.resonant_mask;
    d.use_dk = c->dv.use_dk;
    d.eom = c->dv.eom;
    for (int x = 0; x < 3; x++) {
        d.kappa[x] = c->dv.kappa[x];
        d.bc_re[x] = c->dv.bc_re[x];
        d.bc_im[x] = c->dv.bc_im[x];
        d.outscale[x] = c->dv.outscale[x];
        d.pscale[x] = c->dv.pscale[x];
    }
    d.h = c->dv.h;
    d.eom_beta = c->cavity.eom_beta_rad;
    d.eom_f = c->cavity.eom_f_hz;
    d.t_rt = c->cavity.t_rt_s > 0.0 ? c->cavity.t_rt_s : c->grid.t_window_s;
    d.dt = c->grid.t_window_s / (double)c->n;
    d.t_window = c->grid.t_window_s;
    d.m_start = c->rt;
    d.ns = c->dv.ns;
    d.kerr = c->dv.kerr;
    for (int i = 0; i < 9; i++)
        d.kerr_g[i] = c->dv.kerr_g[i];
    d.cry = c->d_cry;
    d.ncry = c->ncry;
    d.xg1 = c->d_scratch;
    d.xg2 = c->d_xg;
}

int fused_run(opo_ctx *const *ctxs, int count, const FusedCfg &cfg, int64_t m, cudaStream_t s)
{
    const opo_ctx *c0 = ctxs[0];
    const bool dbl = c0->prec == OPO_FP64;
    int fmax = 0, nc_max = 0, lmax = 0;
    std::vector<InstDesc> h(count);
    for (int i = 0; i < count; i++) {
        fill_desc(h[i], ctxs[i]);
        fmax = std::max(fmax, ctxs[i]->F);
        nc_max = std::max(nc_max, ctxs[i]->n / cfg.cluster);
        lmax = std::max(lmax, 1 << std::max(h[i].logP, h[i].logQ));
    }
    // descriptors: a device copy owned by this call, freed stream-ordered
    InstDesc *dd = nullptr;
    if (cudaMallocAsync((void **)&dd, sizeof(InstDesc) * count, s) != cudaSuccess)
        return OPO_E_NOMEM;
    // the pageable source is staged before cudaMemcpyAsync returns
    if (cudaMemcpyAsync(dd, h.data(), sizeof(InstDesc) * count, cudaMemcpyHostToDevice, s) !=
        cudaSuccess)
        return OPO_E_CUDA;
    const size_t sm = cfg.kernel >= 2 ? cfg.smem : smem_bytes(c0->csz, fmax, nc_max, lmax, cfg.disp_in_smem);
    if (cfg.kernel == 1) {
        if (dbl) {
            cudaFuncSetAttribute(k_fused<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
            cudaFuncSetAttribute(k_fused<double>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        } else {
            cudaFuncSetAttribute(k_fused<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
            cudaFuncSetAttribute(k_fused<float>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        }
    }
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3(count * cfg.cluster);
    lc.blockDim = dim3(cfg.threads);
    lc.dynamicSmemBytes = sm;
    lc.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cfg.cluster;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    lc.attrs = at;
    lc.numAttrs = 1;
    int rc = OPO_OK;
    for (int64_t done = 0; done < m && rc == OPO_OK; done += cfg.rt_per_launch) {
        int chunk = (int)std::min<int64_t>(cfg.rt_per_launch, m - done);
        int last = (done + chunk >= m) ? 1 : 0;
        if (cfg.kernel >= 2) {
            rc = fused2_launch(dbl, c0->F, c0->logn, dd, count, cfg, (int)done, chunk, last, s);
            continue;
        }
        cudaError_t e;
        if (dbl)
            e = cudaLaunchKernelEx(&lc, k_fused<double>, (const InstDesc *)dd, (int)done, chunk, last,
                                   (int)cfg.disp_in_smem, fmax, nc_max, lmax);
        else
            e = cudaLaunchKernelEx(&lc, k_fused<float>, (const InstDesc *)dd, (int)done, chunk, last,
                                   (int)cfg.disp_in_smem, fmax, nc_max, lmax);
        if (e != cudaSuccess)
            rc = OPO_E_CUDA;
    }
    if (rc == OPO_OK && m > 0) {
        int64_t work = (int64_t)count * m;
        int nb = (int)std::min<int64_t>((work + 255) / 256, 4096);
        k_finalize_fused<<<nb, 256, 0, s>>>(dd, count, cfg.cluster, (int)m);
        if (cudaGetLastError() != cudaSuccess)
            rc = OPO_E_CUDA;
    }
    cudaFreeAsync(dd, s);
    return rc;
}

} // namespace opo
