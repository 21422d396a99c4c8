// opo_fused2.cu -- configuration and dispatch of the size-specialised fused
// kernel (opo_fused2.cuh); the kernels are instantiated in opo_fused2_*.cu.
#include <algorithm>

#include "opo_fused2.cuh"

namespace opo {
namespace {

int dispatch(int op, bool ip, int nl, bool dbl, int F, int logn, const InstDesc *dd, int count,
             int C, int threads, size_t sm, bool ds, int r_base, int chunk, int last,
             cudaStream_t s)
{
    if (dbl)
        return F == 3 ? f2::dispatch_f64_f3(op, ip, nl, logn, dd, count, C, threads, sm, ds, r_base,
                                            chunk, last, s)
                      : f2::dispatch_f64_f2(op, ip, nl, logn, dd, count, C, threads, sm, ds, r_base,
                                            chunk, last, s);
    return F == 3 ? f2::dispatch_f32_f3(op, ip, nl, logn, dd, count, C, threads, sm, ds, r_base,
                                        chunk, last, s)
                  : f2::dispatch_f32_f2(op, ip, nl, logn, dd, count, C, threads, sm, ds, r_base,
                                        chunk, last, s);
}

// In place with the exchange through global memory: one buffer (X and Y
// alias), three FP32 fields at 2^17 or FP64 at 2^16, 16-CTA clusters.
bool xg_config(bool dbl, int nl, int F, int logn, int C, int threads_req, FusedCfg *out)
{
    if (!((logn == 17 && !dbl) || (logn == 16 && dbl)) || C != 16)
        return false;
    const int LP = logn / 2, LQ = logn - LP;
    const int nc = (1 << logn) / C;
    const size_t csz = dbl ? sizeof(double2) : sizeof(float2);
    const int LS = (logn + 1) / 2;
    // one buffer; stage twiddles (2P + 2Q); W_N halves (lo, hi)
    const size_t el = (size_t)F * nc + 2 * (1 << LP) + 2 * (1 << LQ) + (1 << LS) +
                      ((1 << logn) >> LS);
    const size_t sm = el * csz + 32 * kNslot * sizeof(double);
    if (sm > 227 * 1024)
        return false;
    const int maxT = dbl ? 256 : 384;
    const int threads = threads_req > 0 ? threads_req : 256;
    if (threads < 32 || threads > maxT || (threads & 31))
        return false;
    if (dispatch(1, true, nl, dbl, F, logn, nullptr, 0, C, threads, sm, false, 0, 0, 0, nullptr) < 1)
        return false;
    out->cluster = C;
    out->threads = threads;
    out->disp_in_smem = false;
    out->smem = sm;
    out->kernel = 4;
    out->nl = nl;
    return true;
}

// In-place variant: X and Y only, dispersion factors from L2.
bool ip_config(bool dbl, int nl, int F, int logn, int C, int threads_req, FusedCfg *out)
{
    if (logn < 12 || logn > 16 || (logn == 16 && dbl))
        return false;
    const int LP = logn / 2, LQ = logn - LP;
    if ((1 << LP) < C || (1 << LQ) < C)
        return false;
    const int A2 = f2::f2_col_a2(LP), A1 = LP - A2;
    const int Qc = (1 << LQ) / C;
    const int nc = (1 << logn) / C;
    const int maxT = dbl ? 256
                         : (logn >= 16 ? 384
                                       : (F == 3 && LP == 7 && nl != kNlKerr ? 256
                                                                   : f2::F2IpTraits<float>::kMaxThreads));
    (void)A2;
    const size_t csz = dbl ? sizeof(double2) : sizeof(float2);
    const int LS = (logn + 1) / 2;
    // X, Y; stage twiddles (2P + 2Q); W_N halves (lo, hi)
    size_t el = (size_t)F * nc * 2 + 2 * (1 << LP) + 2 * (1 << LQ) + (1 << LS) +
                ((1 << logn) >> LS);
    size_t sm = el * csz + 32 * kNslot * sizeof(double);
    if (sm > 227 * 1024)
        return false;
    int threads = threads_req;
    if (threads == 0) {
        // one phase-2 item per thread; 2^16: 256 (two block-A items per
        // thread) measured best; three FP32 fields where the shared memory
        // admits two CTAs per SM: 128, so that the registers admit them too
        // (2^14 on 8-CTA clusters 93.7 against 64.7 G point-field-steps/s
        // with 384 threads, 2^15 on 16-CTA clusters 72.3 against 55.8)
        threads = logn >= 16 ? 256 : std::min(maxT, (F * Qc * (1 << A1) + 31) / 32 * 32);
        if (!dbl && F == 3 && logn < 16 && 2 * (sm + 1024) <= 228 * 1024)
            threads = 128;
    }
    if (threads < 32 || threads > maxT || (threads & 31))
        return false;
    if (dispatch(1, true, nl, dbl, F, logn, nullptr, 0, C, threads, sm, false, 0, 0, 0, nullptr) < 1)
        return false;
    out->cluster = C;
    out->threads = threads;
    out->disp_in_smem = false;
    out->smem = sm;
    out->kernel = 3;
    out->nl = nl;
    return true;
}

} // namespace

namespace {

bool three_buffer_config(bool dbl, int nl, int F, int logn, int C, int threads_req,
                         FusedCfg *out)
{
    const int LP = logn / 2, LQ = logn - LP;
    if ((1 << LP) < C || (1 << LQ) < C)
        return false;
    const int A1 = LP - f2::f2_col_a2(LP);
    const int B1 = LQ - (LQ + 1) / 2, B2 = (LQ + 1) / 2;
    const int nc = (1 << logn) / C;
    const int Qc = (1 << LQ) / C, Pc = (1 << LP) / C;
    const size_t csz = dbl ? sizeof(double2) : sizeof(float2);
    const int LS = (logn + 1) / 2;
    const int maxT = dbl ? 256 : 384;
    // default: one work item per thread in the column phases (2 and 6);
    // the row phases may take two rounds
    int items = F * Qc * (1 << A1);
    int threads = threads_req > 0 ? threads_req
                                  : (logn >= 16 ? 256 : std::min(maxT, ((items + 31) / 32) * 32));
    if (threads > maxT || threads < 32 || (threads & 31))
        return false;
    (void)B1;
    (void)B2;
    (void)Pc;
    for (int ds = 1; ds >= 0; ds--) {
        size_t el = (size_t)F * nc * (ds ? 4 : 3) + 2 * (1 << LP) + 2 * (1 << LQ) + (1 << LS) +
                    ((1 << logn) >> LS);
        size_t sm = el * csz + 32 * kNslot * sizeof(double);
        if (sm > 227 * 1024)
            continue;
        if (dispatch(1, false, nl, dbl, F, logn, nullptr, 0, C, threads, sm, ds == 1, 0, 0, 0,
                     nullptr) < 1)
            continue;
        out->cluster = C;
        out->threads = threads;
        out->disp_in_smem = ds == 1;
        out->smem = sm;
        out->kernel = 2;
        out->nl = nl;
        return true;
    }
    return false;
}

} // namespace

// Of the two forms that can run (N, F, C, threads), take the one with more
// clusters co-resident on the device (the in-place form holds twice the
// points per CTA, so where both fit it usually packs two CTAs per SM); on a
// tie the three-buffer form if it keeps the dispersion factors in shared
// memory, else the in-place form (cheaper addressing, same passes).
bool fused2_config(bool dbl, int nl, int F, int logn, int C, int threads_req, FusedCfg *out)
{
    if ((logn == 17 && !dbl) || (logn == 16 && dbl))
        return xg_config(dbl, nl, F, logn, C, threads_req, out);
    if (logn < 12 || logn > 16)
        return false;
    FusedCfg a, b;
    const bool ok_a = three_buffer_config(dbl, nl, F, logn, C, threads_req, &a);
    const bool ok_b = ip_config(dbl, nl, F, logn, C, threads_req, &b);
    if (!ok_a && !ok_b)
        return false;
    if (ok_a && ok_b) {
        const int na = fused2_max_active(dbl, F, logn, a);
        const int nb = fused2_max_active(dbl, F, logn, b);
        *out = (nb > na || (nb == na && !a.disp_in_smem)) ? b : a;
    } else {
        *out = ok_a ? a : b;
    }
    return true;
}

int fused2_max_active(bool dbl, int F, int logn, const FusedCfg &cfg)
{
    return dispatch(1, cfg.kernel >= 3, cfg.nl, dbl, F, logn, nullptr, 0, cfg.cluster,
                    cfg.threads, cfg.smem, cfg.disp_in_smem, 0, 0, 0, nullptr);
}

int fused2_launch(bool dbl, int F, int logn, const InstDesc *dd, int count, const FusedCfg &cfg,
                  int r_base, int chunk, int last, cudaStream_t s)
{
    return dispatch(0, cfg.kernel >= 3, cfg.nl, dbl, F, logn, dd, count, cfg.cluster,
                    cfg.threads, cfg.smem, cfg.disp_in_smem, r_base, chunk, last, s);
}

} // namespace opo
