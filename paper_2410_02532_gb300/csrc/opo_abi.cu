// opo_abi.cu -- the C ABI of libopo.so (declared in include/opo.h): context
// lifecycle, argument validation, device memory, path selection (plain
// per-operation graph or fused persistent cluster kernel), the batched
// sweep, field transfer and the per-round-trip trace.
#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstring>
#include <new>
#include <vector>

#include "opo_common.cuh"
#include "opo_internal.h"

using namespace opo;

namespace {

// Make the context's device current for the duration of a call and restore
// the caller's device afterwards.
struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess)
            prev = -1;
        ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard()
    {
        if (prev >= 0)
            cudaSetDevice(prev);
    }
};

int cuda_status(cudaError_t e)
{
    if (e == cudaSuccess)
        return OPO_OK;
    if (e == cudaErrorMemoryAllocation)
        return OPO_E_NOMEM;
    return OPO_E_CUDA;
}

bool finite_all(const double *v, int k)
{
    for (int i = 0; i < k; i++)
        if (!std::isfinite(v[i]))
            return false;
    return true;
}

bool is_pow2(int64_t v) { return v > 0 && (v & (v - 1)) == 0; }

template <class T>
__global__ void k_from_f64(cv<T> *dst, const double *src, int n)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        dst[i] = cmk<cv<T>>((T)src[2 * i], (T)src[2 * i + 1]);
}

// One member of a batch host transfer.
struct XMember {
    void *fields, *out;   // F*N state and output fields (context precision)
    const double *trace;  // rows {P_p, P_s, P_i, nu_c}
    long long off_all;    // first complex of this member in a [F][N] transfer
    long long off_n;      // first complex of this member in a one-field transfer
    int n, F, dbl;
};

__device__ __forceinline__ int xmember_of(const XMember *m, int count, long long e, bool all)
{
    int lo = 0, hi = count - 1; // last member whose offset is <= e
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if ((all ? m[mid].off_all : m[mid].off_n) <= e)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

__global__ void k_batch_from_f64(const XMember *m, int count, const double *src, long long total)
{
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const XMember &x = m[xmember_of(m, count, e, true)];
        const long long i = e - x.off_all;
        if (x.dbl)
            ((double2 *)x.fields)[i] = make_double2(src[2 * e], src[2 * e + 1]);
        else
            ((float2 *)x.fields)[i] = make_float2((float)src[2 * e], (float)src[2 * e + 1]);
    }
}

__global__ void k_batch_to_f64(const XMember *m, int count, int field, int which, double *dst,
                               long long total)
{
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const XMember &x = m[xmember_of(m, count, e, false)];
        const long long i = (long long)field * x.n + (e - x.off_n);
        double re = 0.0, im = 0.0;
        if (field < x.F) {
            const void *b = which == OPO_OUTPUT ? x.out : x.fields;
            if (x.dbl) {
                const double2 v = ((const double2 *)b)[i];
                re = v.x;
                im = v.y;
            } else {
                const float2 v = ((const float2 *)b)[i];
                re = (double)v.x;
                im = (double)v.y;
            }
        }
        dst[2 * e] = re;
        dst[2 * e + 1] = im;
    }
}

__global__ void k_batch_trace(const XMember *m, int count, int rows, double *dst)
{
    const long long per = 4LL * rows, total = per * count;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x)
        dst[e] = m[e / per].trace[e % per];
}

// Row rows - 1 of every member's trace, members in order (4 doubles each).
__global__ void k_batch_last_row(const XMember *m, int count, int rows, double *dst)
{
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < 4 * count; e += gridDim.x * blockDim.x)
        dst[e] = m[e / 4].trace[4LL * (rows - 1) + e % 4];
}

__global__ void k_gather_err(int *const *src, int count, int *dst)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x)
        dst[i] = *src[i];
}

template <class T>
__global__ void k_to_f64(double *dst, const cv<T> *src, int n)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        cv<T> v = src[i];
        dst[2 * i] = (double)v.x;
        dst[2 * i + 1] = (double)v.y;
    }
}

__global__ void k_ctl_begin(DevCtl *ctl, int64_t rt0, double *obs, int parts)
{
    ctl->rt0 = rt0;
    ctl->slot = 0;
    ctl->obs = obs;
    ctl->parts = parts;
}

int blocks(int64_t work)
{
    int64_t b = (work + 255) / 256;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, 4096));
}

void free_all(opo_ctx *c)
{
    void *bufs[] = {c->d_fields, c->d_out, c->d_scratch, c->d_xg, c->d_pump, c->d_disp, c->d_gdd,
                    c->d_disp_t, c->d_gdd_t,
                    c->d_tw, c->d_ekz, c->d_pump_user, c->d_obs, c->d_trace, c->d_ctl,
                    c->d_stage};
    for (void *b : bufs)
        if (b)
            cudaFree(b);
    for (int k = 1; k < opo::kMaxCry; k++) {
        opo::CrystalState &x = c->xs[k];
        for (void *b : {x.disp, x.disp_t, x.ekz})
            if (b)
                cudaFree(b);
    }
    if (c->d_cry)
        cudaFree(c->d_cry);
    if (c->d_hist)
        cudaFree(c->d_hist);
    if (c->h_pinned)
        cudaFreeHost(c->h_pinned);
    if (c->graph)
        cudaGraphExecDestroy(c->graph);
    if (c->capture_stream)
        cudaStreamDestroy(c->capture_stream);
    if (c->own_stream && c->stream)
        cudaStreamDestroy(c->stream);
}

int derive(opo_ctx *c)
{
    const opo_crystal &k = c->crystal;
    const opo_cavity &v = c->cavity;
    Derived &d = c->dv;
    for (int x = 0; x < 3; x++) {
        d.kappa[x] = (x < c->F) ? 2.0 * kPi * k.deff_mpv / (k.n[x] * k.lambda_m[x]) : 0.0;
        d.pscale[x] = (x < c->F) ? 0.5 * k.n[x] * kEps0 * kC0 * kPi * k.w0_m * k.w0_m : 0.0;
        bool res = (v.resonant_mask >> x) & 1u;
        double r = res ? std::sqrt(v.R[x]) : 1.0;
        d.bc_re[x] = res ? r * std::cos(v.delta_rad[x]) : 1.0;
        d.bc_im[x] = res ? r * std::sin(v.delta_rad[x]) : 0.0;
        d.outscale[x] = res ? std::sqrt(1.0 - v.R[x]) : 1.0;
    }
    d.dz = k.length_m / (double)k.nz;
    d.h = 0.5 * d.dz;
    d.use_dk = k.dk_per_m != 0.0;
    d.eom = v.eom_beta_rad != 0.0;
    d.kerr = kerr_coefficients(k, c->F, d.kerr_g);
    // every crystal's descriptor (device pointers are filled in by the table
    // setup); the specialised kernels take the Kerr instantiation when any
    // crystal has the terms
    c->kerr_any = false;
    c->dk_any = false;
    for (int i = 0; i < c->ncry; i++) {
        const opo_crystal &ki = c->cry[i];
        CryDesc &cd = c->h_cry[i];
        for (int x = 0; x < 3; x++)
            cd.kappa[x] = (x < c->F) ? 2.0 * kPi * ki.deff_mpv / (ki.n[x] * ki.lambda_m[x]) : 0.0;
        cd.h = 0.5 * ki.length_m / (double)ki.nz;
        cd.nz = ki.nz;
        cd.use_dk = ki.dk_per_m != 0.0;
        cd.kerr = kerr_coefficients(ki, c->F, cd.kerr_g);
        for (int x = 0; x < 13; x++)
            cd.kf[x] = (float)(x < 3 ? cd.kappa[x] : x == 3 ? cd.h : cd.kerr_g[x - 4]);
        c->kerr_any = c->kerr_any || cd.kerr;
        c->dk_any = c->dk_any || cd.use_dk;
    }
    d.ns = NsPump{};
    d.ns.n = c->n;
    d.ns.dt = c->grid.t_window_s / (double)c->n;
    d.ns.t_rt = v.t_rt_s > 0.0 ? v.t_rt_s : c->grid.t_window_s;
    if (v.pump_kind == OPO_PUMP_NS) {
        // peak power -> peak field: P = (1/2) n_p eps0 c |A|^2 pi w0^2
        double intensity = v.pump_power_W / (kPi * k.w0_m * k.w0_m);
        d.ns.a0 = std::sqrt(2.0 * intensity / (k.n[0] * kEps0 * kC0));
        d.ns.c = 2.0 * std::log(2.0) / (v.pump_fwhm_s * v.pump_fwhm_s);
        d.ns.t0 = v.pump_t0_s;
        d.ns.on = 1;
    }
    return OPO_OK;
}

int ensure_obs(opo_ctx *c, int64_t M, int parts)
{
    int64_t need = std::max<int64_t>(M, 1);
    if (need <= c->obs_cap && parts <= c->obs_parts_cap)
        return OPO_OK;
    int64_t cap = std::max<int64_t>(need, 2 * c->obs_cap);
    int pc = std::max(parts, c->obs_parts_cap);
    double *o = nullptr, *t = nullptr;
    cudaStreamSynchronize(c->stream);
    if (cudaMalloc((void **)&o, sizeof(double) * cap * pc * kNslot) != cudaSuccess)
        return OPO_E_NOMEM;
    if (cudaMalloc((void **)&t, sizeof(double) * cap * 4) != cudaSuccess) {
        cudaFree(o);
        return OPO_E_NOMEM;
    }
    // keep the previous call's trace readable
    if (c->d_trace)
        cudaMemcpy(t, c->d_trace, sizeof(double) * std::min(c->obs_cap, cap) * 4,
                   cudaMemcpyDeviceToDevice);
    if (c->d_obs)
        cudaFree(c->d_obs);
    if (c->d_trace)
        cudaFree(c->d_trace);
    c->d_obs = o;
    c->d_trace = t;
    c->obs_cap = cap;
    c->obs_parts_cap = pc;
    return OPO_OK;
}

int check_err(opo_ctx *c)
{
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess)
        return OPO_E_CUDA;
    int err = 0;
    if (cudaMemcpy(&err, (char *)c->d_ctl + offsetof(DevCtl, err), sizeof(int),
                   cudaMemcpyDeviceToHost) != cudaSuccess)
        return OPO_E_CUDA;
    // bit 0: a non-finite field; bit 1 (reserved): a bounded device wait gave up
    return err ? ((err & 2) ? OPO_E_TIMEOUT : OPO_E_NONFINITE) : OPO_OK;
}

int build_graph(opo_ctx *c)
{
    if (c->graph_valid)
        return OPO_OK;
    if (c->graph) {
        cudaGraphExecDestroy(c->graph);
        c->graph = nullptr;
    }
    plain_prepare(c);
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(c->capture_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return OPO_E_CUDA;
    int rc = plain_enqueue_roundtrip(c, c->capture_stream);
    cudaError_t e = cudaStreamEndCapture(c->capture_stream, &g);
    if (rc != OPO_OK || e != cudaSuccess) {
        if (g)
            cudaGraphDestroy(g);
        cudaGetLastError();
        return OPO_E_CUDA;
    }
    e = cudaGraphInstantiate(&c->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess)
        return OPO_E_CUDA;
    c->graph_valid = true;
    return OPO_OK;
}

int choose_path(opo_ctx *c, FusedCfg *cfg)
{
    if (c->path_req == OPO_PATH_PLAIN)
        return OPO_PATH_PLAIN;
    bool ok = fused_config(c->csz, c->F, c->F, c->n, c->n, c->cluster_req, c->rtpl_req,
                           c->threads_req, nl_variant(c), cfg);
    if (c->path_req == OPO_PATH_FUSED)
        return ok ? OPO_PATH_FUSED : -1;
    return ok ? OPO_PATH_FUSED : OPO_PATH_PLAIN;
}

// Observable storage for M round trips; the plain path also resets the
// device control block its captured graph reads.
int begin_call(opo_ctx *c, int64_t M, int parts, bool plain)
{
    int rc = ensure_obs(c, M, parts);
    if (rc != OPO_OK || !plain)
        return rc;
    k_ctl_begin<<<1, 1, 0, c->stream>>>(c->d_ctl, c->rt, c->d_obs, parts);
    return cuda_status(cudaGetLastError());
}

} // namespace

namespace opo {

// The grid checks of opo_create that need no device: N a power of two in
// [16, 2^17], a finite positive window, two or three fields, a known
// precision.
bool valid_grid_shape(const opo_grid *g)
{
    if (!is_pow2(g->n) || g->n < 16 || g->n > (1 << 17))
        return false;
    if (!(g->t_window_s > 0.0) || !std::isfinite(g->t_window_s))
        return false;
    if (g->nfields != 2 && g->nfields != 3)
        return false;
    return g->precision == OPO_FP64 || g->precision == OPO_FP32_PH64;
}

// A crystal for F fields: positive finite length, 1..10^6 steps, finite
// parameters, positive wavelengths and indices of the used fields, waist > 0,
// TOD divisor finite and >= 0 (0 selects 6).
bool valid_crystal_for(int F, const opo_crystal *k)
{
    if (!(k->length_m > 0.0) || !std::isfinite(k->length_m) || k->nz < 1 || k->nz > 1000000)
        return false;
    if (!std::isfinite(k->dk_per_m) || !std::isfinite(k->deff_mpv) || !(k->w0_m > 0.0) ||
        !std::isfinite(k->w0_m) || !std::isfinite(k->tod_div) || k->tod_div < 0.0)
        return false;
    if (!finite_all(k->lambda_m, 3) || !finite_all(k->n, 3) || !finite_all(k->alpha_per_m, 3) ||
        !finite_all(k->dbeta1_s_per_m, 3) || !finite_all(k->beta2_s2_per_m, 3) ||
        !finite_all(k->beta3_s3_per_m, 3) || !finite_all(k->beta4_s4_per_m, 3) ||
        !std::isfinite(k->n2_m2_per_W))
        return false;
    for (int x = 0; x < F; x++)
        if (!(k->lambda_m[x] > 0.0) || !(k->n[x] > 0.0))
            return false;
    return true;
}

// A cavity for F fields of N points: resonant bits only for existing fields,
// 0 <= R <= 1, finite phases, GDD, delay, EOM and pump parameters, a known
// pump kind with a positive width where it needs one and a finite user
// profile where it is used.
bool valid_cavity_for(int F, int n, const opo_cavity *v)
{
    if (v->resonant_mask >> F)
        return false;
    for (int x = 0; x < 3; x++)
        if (!(v->R[x] >= 0.0 && v->R[x] <= 1.0))
            return false;
    if (!finite_all(v->delta_rad, 3) || !finite_all(v->gdd_s2, 3) || !std::isfinite(v->delay_s) ||
        !std::isfinite(v->eom_beta_rad) || !std::isfinite(v->eom_f_hz) ||
        !std::isfinite(v->t_rt_s) || v->t_rt_s < 0.0 || !std::isfinite(v->pump_power_W) ||
        v->pump_power_W < 0.0 || !std::isfinite(v->pump_fwhm_s) || !std::isfinite(v->pump_t0_s))
        return false;
    if (v->pump_kind < OPO_PUMP_CW || v->pump_kind > OPO_PUMP_NS)
        return false;
    if ((v->pump_kind == OPO_PUMP_SECH2 || v->pump_kind == OPO_PUMP_NS) && !(v->pump_fwhm_s > 0.0))
        return false;
    if (v->pump_kind == OPO_PUMP_USER) {
        if (!v->pump_user)
            return false;
        if (!finite_all(v->pump_user, 2 * n))
            return false;
    }
    return true;
}

// Crystals of one round trip: each valid for F fields, the same wavelengths
// in all of them.
bool valid_crystals_for(int F, const opo_crystal *list, int count)
{
    if (!list || count < 1 || count > OPO_MAX_CRYSTALS)
        return false;
    for (int i = 0; i < count; i++) {
        if (!valid_crystal_for(F, &list[i]))
            return false;
        for (int x = 0; x < F; x++)
            if (list[i].lambda_m[x] != list[0].lambda_m[x])
                return false; // the same fields in every crystal
    }
    return true;
}

} // namespace opo

extern "C" {

int opo_validate(const opo_grid *grid, const opo_crystal *crystals, int32_t count,
                 const opo_cavity *cavity)
{
    if (!grid || !valid_grid_shape(grid) || count < 0)
        return OPO_E_INVALID;
    if (count > 0 && !valid_crystals_for(grid->nfields, crystals, count))
        return OPO_E_INVALID;
    if (cavity && !valid_cavity_for(grid->nfields, grid->n, cavity))
        return OPO_E_INVALID;
    return OPO_OK;
}

const char *opo_status_string(int s)
{
    switch (s) {
    case OPO_OK: return "ok";
    case OPO_E_INVALID: return "invalid argument";
    case OPO_E_NOMEM: return "device allocation failed";
    case OPO_E_CUDA: return "CUDA runtime error";
    case OPO_E_NONFINITE: return "non-finite field (step dz too large?)";
    case OPO_E_TIMEOUT: return "device wait timed out";
    case OPO_E_STATE: return "call out of order (crystal or cavity not set)";
    case OPO_E_UNSUPPORTED: return "unsupported by the requested path";
    default: return "unknown status";
    }
}

int opo_create(opo_ctx **out, const opo_grid *grid)
{
    if (!out)
        return OPO_E_INVALID;
    *out = nullptr;
    if (!grid)
        return OPO_E_INVALID;
    if (!valid_grid_shape(grid))
        return OPO_E_INVALID;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return OPO_E_CUDA;
    }
    if (grid->device < 0 || grid->device >= ndev)
        return OPO_E_INVALID;
    DeviceGuard g(grid->device);
    if (!g.ok)
        return OPO_E_CUDA;
    opo_ctx *c = new (std::nothrow) opo_ctx();
    if (!c)
        return OPO_E_NOMEM;
    c->grid = *grid;
    c->device = grid->device;
    c->n = grid->n;
    c->logn = ilog2((unsigned)grid->n);
    c->F = grid->nfields;
    c->prec = grid->precision;
    c->csz = c->prec == OPO_FP64 ? sizeof(double2) : sizeof(float2);
    int rc = OPO_OK;
    auto alloc = [&](void **p, size_t bytes) {
        if (rc != OPO_OK)
            return;
        cudaError_t e = cudaMalloc(p, bytes);
        if (e != cudaSuccess)
            rc = cuda_status(e);
    };
    const size_t fb = c->csz * (size_t)c->F * c->n;
    alloc(&c->d_fields, fb);
    alloc(&c->d_out, fb);
    alloc(&c->d_scratch, fb);
    // the sizes whose fused form exchanges through global memory need a
    // second exchange buffer
    if ((c->prec == OPO_FP32_PH64 && c->n == (1 << 17)) || (c->prec == OPO_FP64 && c->n == (1 << 16)))
        alloc(&c->d_xg, fb);
    alloc(&c->d_disp, fb);
    alloc(&c->d_gdd, fb);
    alloc(&c->d_disp_t, fb);
    alloc(&c->d_gdd_t, fb);
    alloc(&c->d_pump, c->csz * c->n);
    alloc(&c->d_tw, c->csz * c->n);
    alloc((void **)&c->d_pump_user, sizeof(double) * 2 * c->n);
    alloc((void **)&c->d_stage, sizeof(double) * 2 * c->n);
    alloc((void **)&c->d_ctl, sizeof(DevCtl));
    if (rc == OPO_OK) {
        if (grid->stream) {
            c->stream = (cudaStream_t)grid->stream;
        } else {
            rc = cuda_status(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
            c->own_stream = rc == OPO_OK;
        }
    }
    if (rc == OPO_OK)
        rc = cuda_status(cudaStreamCreateWithFlags(&c->capture_stream, cudaStreamNonBlocking));
    if (rc == OPO_OK) {
        cudaMemsetAsync(c->d_fields, 0, fb, c->stream);
        cudaMemsetAsync(c->d_out, 0, fb, c->stream);
        cudaMemsetAsync(c->d_ctl, 0, sizeof(DevCtl), c->stream);
        rc = setup_twiddles(c);
    }
    if (rc == OPO_OK)
        rc = cuda_status(cudaStreamSynchronize(c->stream));
    if (rc != OPO_OK) {
        free_all(c);
        delete c;
        return rc;
    }
    *out = c;
    return OPO_OK;
}

int opo_destroy(opo_ctx *c)
{
    if (!c)
        return OPO_OK;
    DeviceGuard g(c->device);
    if (c->stream)
        cudaStreamSynchronize(c->stream);
    free_all(c);
    delete c;
    return OPO_OK;
}

// Make *p hold at least bytes (re-allocating after the stream drained).
static int ensure_buf(opo_ctx *c, void **p, int *cap, int want, size_t elem)
{
    if (*p && (!cap || want <= *cap))
        return OPO_OK;
    cudaStreamSynchronize(c->stream);
    if (*p)
        cudaFree(*p);
    *p = nullptr;
    if (cap)
        *cap = 0;
    if (cudaMalloc(p, elem * (size_t)want) != cudaSuccess) {
        *p = nullptr;
        return OPO_E_NOMEM;
    }
    if (cap)
        *cap = want;
    return OPO_OK;
}

int opo_set_crystals(opo_ctx *c, const opo_crystal *list, int32_t count)
{
    if (!c || !valid_crystals_for(c->F, list, count))
        return OPO_E_INVALID;
    DeviceGuard g(c->device);
    if (!g.ok)
        return OPO_E_CUDA;
    // device buffers first, so that a failure leaves the old crystals intact
    int rc = ensure_buf(c, &c->d_ekz, &c->ekz_cap, 4 * list[0].nz + 1, c->csz);
    const size_t fb = c->csz * (size_t)c->F * c->n;
    for (int i = 1; i < count && rc == OPO_OK; i++) {
        opo::CrystalState &x = c->xs[i];
        rc = ensure_buf(c, &x.disp, nullptr, 1, fb);
        if (rc == OPO_OK)
            rc = ensure_buf(c, &x.disp_t, nullptr, 1, fb);
        if (rc == OPO_OK)
            rc = ensure_buf(c, &x.ekz, &x.ekz_cap, 4 * list[i].nz + 1, c->csz);
    }
    if (rc == OPO_OK && !c->d_cry)
        rc = ensure_buf(c, (void **)&c->d_cry, nullptr, 1, sizeof(opo::CryDesc) * opo::kMaxCry);
    if (rc != OPO_OK)
        return rc;
    for (int i = 0; i < count; i++)
        c->cry[i] = list[i];
    c->crystal = list[0];
    c->ncry = count;
    c->have_crystal = true;
    c->graph_valid = false;
    c->gen++;
    derive(c);
    rc = setup_crystal_tables(c);
    if (rc == OPO_OK && c->have_cavity)
        rc = setup_cavity_tables(c); // pump amplitude depends on n_p and w0
    return rc;
}

int opo_set_crystal(opo_ctx *c, const opo_crystal *k)
{
    if (!c || !k)
        return OPO_E_INVALID;
    return opo_set_crystals(c, k, 1);
}

int opo_set_cavity(opo_ctx *c, const opo_cavity *v)
{
    if (!c || !v)
        return OPO_E_INVALID;
    if (!valid_cavity_for(c->F, c->n, v))
        return OPO_E_INVALID;
    DeviceGuard g(c->device);
    if (!g.ok)
        return OPO_E_CUDA;
    c->cavity = *v;
    c->cavity.pump_user = nullptr;
    if (v->pump_kind == OPO_PUMP_USER) {
        if (cudaMemcpyAsync(c->d_pump_user, v->pump_user, sizeof(double) * 2 * c->n,
                            cudaMemcpyHostToDevice, c->stream) != cudaSuccess)
            return OPO_E_CUDA;
    }
    c->have_cavity = true;
    c->graph_valid = false;
    c->gen++;
    if (c->have_crystal) {
        derive(c);
        return setup_cavity_tables(c);
    }
    return OPO_OK;
}

static int set_fields_impl(opo_ctx *c, int32_t field, const void *src, size_t n, int64_t rt_index,
                           bool device_src)
{
    if (!c || !src || field < 0 || field >= c->F || n != (size_t)c->n)
        return OPO_E_INVALID;
    DeviceGuard g(c->device);
    if (!g.ok)
        return OPO_E_CUDA;
    char *dst = (char *)c->d_fields + (size_t)field * c->n * c->csz;
    cudaError_t e;
    if (device_src) {
        e = cudaMemcpyAsync(dst, src, c->csz * n, cudaMemcpyDeviceToDevice, c->stream);
    } else {
        e = cudaMemcpyAsync(c->d_stage, src, sizeof(double) * 2 * n, cudaMemcpyHostToDevice,
                            c->stream);
        if (e == cudaSuccess) {
            if (c->prec == OPO_FP64)
                k_from_f64<double><<<blocks(c->n), 256, 0, c->stream>>>((double2 *)dst, c->d_stage, c->n);
            else
                k_from_f64<float><<<blocks(c->n), 256, 0, c->stream>>>((float2 *)dst, c->d_stage, c->n);
            e = cudaGetLastError();
        }
        // the host buffer must be free to reuse when we return
        if (e == cudaSuccess)
            e = cudaStreamSynchronize(c->stream);
    }
    if (e != cudaSuccess)
        return OPO_E_CUDA;
    if (rt_index >= 0) {
        // a new start: round-trip counter and the sticky non-finite flag
        c->rt = rt_index;
        if (cudaMemsetAsync((char *)c->d_ctl + offsetof(DevCtl, err), 0, sizeof(int), c->stream) !=
            cudaSuccess)
            return OPO_E_CUDA;
    }
    return OPO_OK;
}

int opo_set_fields(opo_ctx *c, int32_t field, const double *interleaved, size_t n, int64_t rt_index)
{
    return set_fields_impl(c, field, interleaved, n, rt_index, false);
}

int opo_set_fields_device(opo_ctx *c, int32_t field, const void *dev, size_t n, int64_t rt_index)
{
    return set_fields_impl(c, field, dev, n, rt_index, true);
}

static int get_fields_impl(opo_ctx *c, int32_t field, int32_t which, void *dst, size_t n,
                           bool device_dst)
{
    if (!c || !dst || field < 0 || field >= c->F || n != (size_t)c->n)
        return OPO_E_INVALID;
    if (which != OPO_INTRACAVITY && which != OPO_OUTPUT)
        return OPO_E_INVALID;
    DeviceGuard g(c->device);
    if (!g.ok)
        return OPO_E_CUDA;
    const char *src = (const char *)(which == OPO_OUTPUT ? c->d_out : c->d_fields) +
                      (size_t)field * c->n * c->csz;
    if (device_dst) {
        if (cudaMemcpyAsync(dst, src, c->csz * n, cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess)
            return OPO_E_CUDA;
        return OPO_OK;
    }
    if (c->prec == OPO_FP64)
        k_to_f64<double><<<blocks(c->n), 256, 0, c->stream>>>(c->d_stage, (const double2 *)src, c->n);
    else
        k_to_f64<float><<<blocks(c->n), 256, 0, c->stream>>>(c->d_stage, (const float2 *)src, c->n);
    if (cudaGetLastError() != cudaSuccess)
        return OPO_E_CUDA;
    if (cudaMemcpyAsync(dst, c->d_stage, sizeof(double) * 2 * n, cudaMemcpyDeviceToHost,
                        c->stream) != cudaSuccess)
        return OPO_E_CUDA;
    return check_err(c);
}

int opo_get_fields(opo_ctx *c, int32_t field, int32_t which, double *out, size_t n)
{
    return get_fields_impl(c, field, which, out, n, false);
}

int opo_get_fields_device(opo_ctx *c, int32_t field, int32_t which, void *dev, size_t n)
{
    return get_fields_impl(c, field, which, dev, n, true);
}

int opo_set_path(opo_ctx *c, int32_t path, int32_t cluster, int32_t rt_per_launch,
                 int32_t threads)
{
    if (!c || path < OPO_PATH_AUTO || path > OPO_PATH_FUSED)
        return OPO_E_INVALID;
    if (cluster < 0 || cluster > 16 || (cluster > 0 && !is_pow2(cluster)) || rt_per_launch < 0 ||
        threads < 0 || threads > 1024 || (threads & 31))
        return OPO_E_INVALID;
    if (path == OPO_PATH_FUSED) {
        FusedCfg cfg;
        DeviceGuard g(c->device);
        if (!fused_config(c->csz, c->F, c->F, c->n, c->n, cluster, rt_per_launch, threads,
                          nl_variant(c), &cfg))
            return OPO_E_UNSUPPORTED;
    }
    c->path_req = path;
    c->cluster_req = cluster;
    c->rtpl_req = rt_per_launch;
    c->threads_req = threads;
    return OPO_OK;
}

int opo_set_output_history(opo_ctx *c, int64_t max_rt)
{
    if (!c || max_rt < 0)
        return OPO_E_INVALID;
    const size_t row = c->csz * (size_t)c->F * c->n;
    if (max_rt > (int64_t)(((size_t)1 << 38) / row)) // 256 GiB
        return OPO_E_INVALID;
    DeviceGuard g(c->device);
    if (!g.ok)
        return OPO_E_CUDA;
    cudaStreamSynchronize(c->stream);
    if (c->d_hist)
        cudaFree(c->d_hist);
    c->d_hist = nullptr;
    c->hist_cap = 0;
    c->graph_valid = false;
    c->gen++;
    if (max_rt == 0)
        return OPO_OK;
    if (cudaMalloc(&c->d_hist, row * (size_t)max_rt) != cudaSuccess) {
        c->d_hist = nullptr;
        cudaGetLastError();
        return OPO_E_NOMEM;
    }
    c->hist_cap = max_rt;
    return OPO_OK;
}

int opo_get_output_history(opo_ctx *c, int32_t field, int64_t row0, int64_t rows, double *out)
{
    if (!c || !out || field < 0 || field >= c->F || row0 < 0 || rows < 0)
        return OPO_E_INVALID;
    if (!c->d_hist)
        return OPO_E_STATE;
    if (row0 + rows > c->hist_cap)
        return OPO_E_INVALID;
    DeviceGuard g(c->device);
    if (!g.ok)
        return OPO_E_CUDA;
    for (int64_t r = 0; r < rows; r++) {
        const char *src = (const char *)c->d_hist +
                          ((size_t)(row0 + r) * c->F + field) * (size_t)c->n * c->csz;
        if (c->prec == OPO_FP64)
            k_to_f64<double><<<blocks(c->n), 256, 0, c->stream>>>(c->d_stage, (const double2 *)src, c->n);
        else
            k_to_f64<float><<<blocks(c->n), 256, 0, c->stream>>>(c->d_stage, (const float2 *)src, c->n);
        if (cudaGetLastError() != cudaSuccess)
            return OPO_E_CUDA;
        if (cudaMemcpyAsync(out + (size_t)r * 2 * c->n, c->d_stage, sizeof(double) * 2 * c->n,
                            cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
            return OPO_E_CUDA;
    }
    return check_err(c);
}

int opo_run_roundtrips(opo_ctx *c, int64_t m, opo_stats *stats)
{
    if (!c || m < 0)
        return OPO_E_INVALID;
    if (c->d_hist && m > c->hist_cap)
        return OPO_E_INVALID;
    if (!c->have_crystal || !c->have_cavity)
        return OPO_E_STATE;
    DeviceGuard g(c->device);
    if (!g.ok)
        return OPO_E_CUDA;
    FusedCfg cfg{};
    int path = choose_path(c, &cfg);
    if (path < 0)
        return OPO_E_UNSUPPORTED;
    int parts = path == OPO_PATH_FUSED ? cfg.cluster : 1;
    int rc = begin_call(c, m, parts, path == OPO_PATH_PLAIN);
    if (rc != OPO_OK)
        return rc;
    if (path == OPO_PATH_PLAIN) {
        rc = build_graph(c);
        for (int64_t i = 0; i < m && rc == OPO_OK; i++)
            rc = cuda_status(cudaGraphLaunch(c->graph, c->stream));
        if (rc == OPO_OK)
            rc = finalize_trace(c, m, parts);
    } else if (m > 0) {
        opo_ctx *one[1] = {c};
        rc = fused_run(one, 1, cfg, m, c->stream);
    }
    if (rc != OPO_OK)
        return rc;
    c->rt += m;
    c->last_M = m;
    c->last_parts = parts;
    c->last_path = path;
    c->last_cluster = path == OPO_PATH_FUSED ? cfg.cluster : 0;
    if (!stats)
        return OPO_OK;
    std::memset(stats, 0, sizeof(*stats));
    stats->rt_done = c->rt;
    stats->path = path;
    stats->cluster = c->last_cluster;
    rc = check_err(c);
    if (m > 0) {
        std::vector<double> tr((size_t)m * 4);
        if (cudaMemcpy(tr.data(), c->d_trace, sizeof(double) * 4 * m, cudaMemcpyDeviceToHost) !=
            cudaSuccess)
            return OPO_E_CUDA;
        int64_t K = std::max<int64_t>(10, (m + 9) / 10);
        K = std::min(K, m);
        for (int x = 0; x < 3; x++) {
            stats->p_out_W[x] = tr[(size_t)(m - 1) * 4 + x];
            double s = 0.0;
            for (int64_t r = m - K; r < m; r++)
                s += tr[(size_t)r * 4 + x];
            stats->p_out_mean_W[x] = s / (double)K;
        }
        stats->centroid_hz = tr[(size_t)(m - 1) * 4 + 3];
        double s = 0.0;
        for (int64_t r = m - K; r < m; r++)
            s += tr[(size_t)r * 4 + 3];
        stats->centroid_mean_hz = s / (double)K;
    }
    return rc;
}

int opo_get_trace(opo_ctx *c, double *out, int64_t rows)
{
    if (!c || !out || rows < 0 || rows > c->last_M)
        return OPO_E_INVALID;
    DeviceGuard g(c->device);
    int rc = check_err(c);
    if (rows > 0 &&
        cudaMemcpy(out, c->d_trace, sizeof(double) * 4 * rows, cudaMemcpyDeviceToHost) != cudaSuccess)
        return OPO_E_CUDA;
    return rc;
}

int opo_fused_capacity(const opo_ctx *c, int32_t cluster, int32_t threads, int32_t *max_active,
                       int32_t *cluster_out)
{
    if (!c || !max_active || cluster < 0 || cluster > 16 || (cluster > 0 && !is_pow2(cluster)) ||
        threads < 0 || (threads & 31))
        return OPO_E_INVALID;
    DeviceGuard g(c->device);
    if (!g.ok)
        return OPO_E_CUDA;
    FusedCfg cfg;
    if (!fused_config(c->csz, c->F, c->F, c->n, c->n, cluster, 0, threads, nl_variant(c), &cfg))
        return OPO_E_UNSUPPORTED;
    *max_active = fused_max_active(c->prec == OPO_FP64, c->F, c->n, cfg);
    if (cluster_out)
        *cluster_out = cfg.cluster;
    return OPO_OK;
}

int opo_sync(opo_ctx *c)
{
    if (!c)
        return OPO_E_INVALID;
    DeviceGuard g(c->device);
    return check_err(c);
}

} // extern "C"

// A batch is split into groups.  A fused group holds instances of equal
// (N, field count, nonlinear-step variant, launch shape) and runs as one
// fused launch with the configuration a lone instance of that group would
// get; a plain group holds instances of equal (N, field count, crystals'
// step counts) on the plain path and runs one launch per operation for all of
// them (a captured graph per round trip).  Either way every instance advances
// bit-for-bit as it would alone.  Groups run concurrently on forked streams.
struct BatchGroup {
    std::vector<opo_ctx *> ctxs;
    FusedCfg cfg{};
    bool plain = false;
    std::vector<int> nzs;              // plain: every crystal's step count
    opo::PlainInst *d_insts = nullptr; // plain: member descriptors (device)
    opo::PlainCall *d_calls = nullptr; // plain: per-call values (device)
    std::vector<opo::PlainInst> h_insts;
    cudaGraphExec_t graph = nullptr;   // plain: one round trip of every member
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
};

struct opo_batch {
    std::vector<opo_ctx *> ctxs;
    std::vector<BatchGroup> groups;
    cudaStream_t capture = nullptr; // capture of the plain groups' graphs
    bool one_launch = false;        // all fused members in one launch
    std::vector<cudaEvent_t> ev; // one per context: stream ordering
    cudaEvent_t fork = nullptr;
    int device = 0;              // copies, so that destroying the batch never
    cudaStream_t stream = nullptr; // reads a member context
    // host transfers of the whole batch (allocated on first use)
    double *d_xfer = nullptr;    // staging, FP64 interleaved
    size_t xfer_cap = 0;         // doubles
    XMember *d_mem = nullptr;    // member table of the transfer kernels
    std::vector<XMember> h_mem;
    std::vector<XMember> h_mem_dev; // what d_mem holds
    int **d_err = nullptr;       // members' sticky error words
    int *d_errs = nullptr;       // their copies, one per member
    // overlapped host transfers (opo_batch_step_io): two slots each way
    cudaStream_t io_in = nullptr, io_out = nullptr;
    double *d_in[2] = {nullptr, nullptr}, *d_out[2] = {nullptr, nullptr};
    cudaEvent_t ev_h2d[2] = {nullptr, nullptr};  // staged input copied in
    cudaEvent_t ev_used[2] = {nullptr, nullptr}; // staged input consumed
    cudaEvent_t ev_gath[2] = {nullptr, nullptr}; // output gathered
    cudaEvent_t ev_d2h[2] = {nullptr, nullptr};  // output copied out
    int io_slot = 0;
};

static void batch_free(opo_batch *b)
{
    for (void *p : {(void *)b->d_xfer, (void *)b->d_err, (void *)b->d_errs, (void *)b->d_mem,
                    (void *)b->d_in[0], (void *)b->d_in[1], (void *)b->d_out[0],
                    (void *)b->d_out[1]})
        if (p)
            cudaFree(p);
    for (int k = 0; k < 2; k++)
        for (cudaEvent_t e : {b->ev_h2d[k], b->ev_used[k], b->ev_gath[k], b->ev_d2h[k]})
            if (e)
                cudaEventDestroy(e);
    for (cudaStream_t st : {b->io_in, b->io_out})
        if (st)
            cudaStreamDestroy(st);
    for (BatchGroup &g : b->groups) {
        if (g.stream)
            cudaStreamDestroy(g.stream);
        if (g.done)
            cudaEventDestroy(g.done);
        if (g.graph)
            cudaGraphExecDestroy(g.graph);
        if (g.d_insts)
            cudaFree(g.d_insts);
        if (g.d_calls)
            cudaFree(g.d_calls);
    }
    if (b->capture)
        cudaStreamDestroy(b->capture);
    for (cudaEvent_t e : b->ev)
        if (e)
            cudaEventDestroy(e);
    if (b->fork)
        cudaEventDestroy(b->fork);
    delete b;
}

extern "C" {

int opo_batch_create(opo_batch **out, opo_ctx *const *ctxs, int32_t count, int32_t cluster,
                     int32_t threads)
{
    if (!out)
        return OPO_E_INVALID;
    *out = nullptr;
    if (!ctxs || count < 1)
        return OPO_E_INVALID;
    if (cluster < 0 || cluster > 16 || (cluster > 0 && !is_pow2(cluster)) || threads < 0 ||
        (threads & 31))
        return OPO_E_INVALID;
    for (int i = 0; i < count; i++) {
        const opo_ctx *c = ctxs[i];
        if (!c)
            return OPO_E_INVALID;
        if (c->device != ctxs[0]->device || c->prec != ctxs[0]->prec)
            return OPO_E_INVALID;
        if (!c->have_crystal || !c->have_cavity)
            return OPO_E_STATE;
        for (int j = 0; j < i; j++)
            if (ctxs[j] == c)
                return OPO_E_INVALID;
    }
    DeviceGuard g(ctxs[0]->device);
    if (!g.ok)
        return OPO_E_CUDA;
    opo_batch *b = new (std::nothrow) opo_batch();
    if (!b)
        return OPO_E_NOMEM;
    b->ctxs.assign(ctxs, ctxs + count);
    b->device = ctxs[0]->device;
    b->stream = ctxs[0]->stream;
    // launch shape of a context: the batch's arguments where nonzero, else the
    // context's own opo_set_path request
    auto want = [&](const opo_ctx *c, int *cl, int *th, int *rt) {
        *cl = cluster > 0 ? cluster : c->cluster_req;
        *th = threads > 0 ? threads : c->threads_req;
        *rt = c->rtpl_req;
    };
    auto crystal_steps = [](const opo_ctx *c) {
        std::vector<int> v;
        for (int k = 0; k < c->ncry; k++)
            v.push_back(c->cry[k].nz);
        return v;
    };
    for (int i = 0; i < count; i++) {
        opo_ctx *c = ctxs[i];
        int cl, th, rt;
        want(c, &cl, &th, &rt);
        // the path: a plain request, or a size the fused kernels cannot hold
        // with the automatic choice, runs in a plain group
        FusedCfg fc{};
        bool plain = c->path_req == OPO_PATH_PLAIN;
        if (!plain && !fused_config(c->csz, c->F, c->F, c->n, c->n, cl, rt, th, nl_variant(c), &fc)) {
            if (c->path_req == OPO_PATH_FUSED) {
                batch_free(b);
                return OPO_E_UNSUPPORTED;
            }
            plain = true;
        }
        int gi = -1;
        for (size_t k = 0; k < b->groups.size() && gi < 0; k++) {
            const BatchGroup &gg = b->groups[k];
            const opo_ctx *g0 = gg.ctxs[0];
            if (gg.plain != plain || g0->n != c->n || g0->F != c->F)
                continue;
            if (plain) {
                if (gg.nzs == crystal_steps(c))
                    gi = (int)k;
                continue;
            }
            int cl0, th0, rt0;
            want(g0, &cl0, &th0, &rt0);
            if (nl_variant(g0) == nl_variant(c) && cl0 == cl && th0 == th && rt0 == rt)
                gi = (int)k;
        }
        if (gi < 0) {
            b->groups.emplace_back();
            gi = (int)b->groups.size() - 1;
            BatchGroup &gg = b->groups[gi];
            gg.plain = plain;
            if (plain)
                gg.nzs = crystal_steps(c);
            else
                gg.cfg = fc;
        }
        b->groups[gi].ctxs.push_back(c);
    }
    int rc = OPO_OK;
    b->ev.assign(count, nullptr);
    for (int i = 0; i < count && rc == OPO_OK; i++)
        rc = cuda_status(cudaEventCreateWithFlags(&b->ev[i], cudaEventDisableTiming));
    if (rc == OPO_OK)
        rc = cuda_status(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming));
    if (b->groups.size() > 1) {
        for (BatchGroup &gg : b->groups) {
            if (rc != OPO_OK)
                break;
            rc = cuda_status(cudaStreamCreateWithFlags(&gg.stream, cudaStreamNonBlocking));
            if (rc == OPO_OK)
                rc = cuda_status(cudaEventCreateWithFlags(&gg.done, cudaEventDisableTiming));
        }
    }
    for (BatchGroup &gg : b->groups) {
        if (rc != OPO_OK || !gg.plain)
            continue;
        const size_t k = gg.ctxs.size();
        rc = cuda_status(cudaMalloc((void **)&gg.d_insts, sizeof(opo::PlainInst) * k));
        if (rc == OPO_OK)
            rc = cuda_status(cudaMalloc((void **)&gg.d_calls, sizeof(opo::PlainCall) * k));
        if (rc == OPO_OK && !b->capture)
            rc = cuda_status(cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking));
    }
    if (rc != OPO_OK) {
        batch_free(b);
        return rc;
    }
    *out = b;
    return OPO_OK;
}

namespace {

// Order the batch's stream after every member's stream (in) or every
// member's stream after the batch's (out).
void batch_fence(opo_batch *b, cudaStream_t s, bool in)
{
    for (size_t i = 0; i < b->ctxs.size(); i++) {
        opo_ctx *c = b->ctxs[i];
        if (c->stream == s)
            continue;
        cudaEventRecord(b->ev[i], in ? c->stream : s);
        cudaStreamWaitEvent(in ? s : c->stream, b->ev[i], 0);
    }
}

int batch_staging(opo_batch *b, size_t doubles)
{
    if (doubles <= b->xfer_cap)
        return OPO_OK;
    cudaStreamSynchronize(b->stream);
    if (b->d_xfer)
        cudaFree(b->d_xfer);
    b->d_xfer = nullptr;
    b->xfer_cap = 0;
    if (cudaMalloc((void **)&b->d_xfer, sizeof(double) * doubles) != cudaSuccess) {
        cudaGetLastError();
        return OPO_E_NOMEM;
    }
    b->xfer_cap = doubles;
    return OPO_OK;
}

// Upload the member table (pointers can change: the trace grows with M).
int batch_members(opo_batch *b, cudaStream_t s)
{
    const int count = (int)b->ctxs.size();
    if (!b->d_mem && cudaMalloc((void **)&b->d_mem, sizeof(XMember) * count) != cudaSuccess) {
        b->d_mem = nullptr;
        cudaGetLastError();
        return OPO_E_NOMEM;
    }
    b->h_mem.resize(count);
    long long oa = 0, on = 0;
    for (int i = 0; i < count; i++) {
        const opo_ctx *c = b->ctxs[i];
        XMember &x = b->h_mem[i];
        x.fields = c->d_fields;
        x.out = c->d_out;
        x.trace = c->d_trace;
        x.off_all = oa;
        x.off_n = on;
        x.n = c->n;
        x.F = c->F;
        x.dbl = c->prec == OPO_FP64;
        oa += (long long)c->F * c->n;
        on += c->n;
    }
    // unchanged since the last upload (the usual case between steps of the
    // same length): nothing to copy
    if (b->h_mem_dev.size() == b->h_mem.size() &&
        std::memcmp(b->h_mem_dev.data(), b->h_mem.data(), sizeof(XMember) * count) == 0)
        return OPO_OK;
    // the pageable source is staged before cudaMemcpyAsync returns
    if (cudaMemcpyAsync(b->d_mem, b->h_mem.data(), sizeof(XMember) * count,
                        cudaMemcpyHostToDevice, s) != cudaSuccess)
        return OPO_E_CUDA;
    b->h_mem_dev = b->h_mem;
    return OPO_OK;
}

int xblocks(long long work)
{
    long long g = (work + 255) / 256;
    return (int)std::max<long long>(1, std::min<long long>(g, 4096));
}

// Wait for the batch's stream, then OPO_E_NONFINITE if any member has set
// its error word (one gather, one copy).
int batch_check_err(opo_batch *b)
{
    const int count = (int)b->ctxs.size();
    if (!b->d_err) {
        std::vector<int *> p(count);
        for (int i = 0; i < count; i++)
            p[i] = (int *)((char *)b->ctxs[i]->d_ctl + offsetof(DevCtl, err));
        if (cudaMalloc((void **)&b->d_err, sizeof(int *) * count) != cudaSuccess ||
            cudaMalloc((void **)&b->d_errs, sizeof(int) * count) != cudaSuccess) {
            cudaGetLastError();
            return OPO_E_NOMEM;
        }
        if (cudaMemcpy(b->d_err, p.data(), sizeof(int *) * count, cudaMemcpyHostToDevice) !=
            cudaSuccess)
            return OPO_E_CUDA;
    }
    k_gather_err<<<1, 256, 0, b->stream>>>(b->d_err, count, b->d_errs);
    std::vector<int> e(count);
    if (cudaMemcpyAsync(e.data(), b->d_errs, sizeof(int) * count, cudaMemcpyDeviceToHost,
                        b->stream) != cudaSuccess)
        return OPO_E_CUDA;
    if (cudaStreamSynchronize(b->stream) != cudaSuccess)
        return OPO_E_CUDA;
    int any = 0;
    for (int v : e)
        any |= v;
    return any ? ((any & 2) ? OPO_E_TIMEOUT : OPO_E_NONFINITE) : OPO_OK;
}

// A member's state no longer matches the group it was put in (its crystals
// or path request changed after the batch was made).
// In one-launch mode a fused group runs the union of its members' nonlinear
// variants (a member may then sit in a more general kernel than alone).
bool group_stale(const BatchGroup &gg, bool one_launch)
{
    for (const opo_ctx *c : gg.ctxs) {
        if (gg.plain) {
            if (c->path_req == OPO_PATH_FUSED || c->ncry != (int)gg.nzs.size())
                return true;
            for (int k = 0; k < c->ncry; k++)
                if (c->cry[k].nz != gg.nzs[k])
                    return true;
        } else if (c->path_req == OPO_PATH_PLAIN) {
            return true;
        } else if (one_launch) {
            const int v = nl_variant(c);
            if (gg.cfg.kernel >= 2 && v != gg.cfg.nl && gg.cfg.nl != kNlKerr &&
                !(gg.cfg.nl == kNlChi2 && v == kNlChi2NoDk))
                return true;
        } else if (nl_variant(c) != gg.cfg.nl) {
            return true;
        }
    }
    return false;
}

// m round trips of a plain group on stream s: member descriptors (uploaded
// when they changed), the per-call start, the captured round trip replayed m
// times, the trace rows.
int run_plain_group(opo_batch *b, BatchGroup &gg, int64_t m, cudaStream_t s)
{
    const int count = (int)gg.ctxs.size();
    std::vector<opo::PlainInst> h(count);
    for (int i = 0; i < count; i++)
        plain_fill_inst(h[i], gg.ctxs[i]);
    if (h.size() != gg.h_insts.size() ||
        std::memcmp(h.data(), gg.h_insts.data(), sizeof(opo::PlainInst) * count) != 0) {
        // the pageable source is staged before cudaMemcpyAsync returns
        if (cudaMemcpyAsync(gg.d_insts, h.data(), sizeof(opo::PlainInst) * count,
                            cudaMemcpyHostToDevice, s) != cudaSuccess)
            return OPO_E_CUDA;
        gg.h_insts = h;
    }
    std::vector<opo::PlainCall> calls(count);
    for (int i = 0; i < count; i++)
        plain_fill_call(calls[i], gg.ctxs[i]);
    if (cudaMemcpyAsync(gg.d_calls, calls.data(), sizeof(opo::PlainCall) * count,
                        cudaMemcpyHostToDevice, s) != cudaSuccess)
        return OPO_E_CUDA;
    int rc = plain_batch_begin(gg.d_calls, count, s);
    if (rc == OPO_OK && !gg.graph) {
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
            return OPO_E_CUDA;
        rc = plain_batch_enqueue_roundtrip(gg.ctxs[0], gg.d_insts, count, b->capture);
        cudaError_t e = cudaStreamEndCapture(b->capture, &g);
        if (rc == OPO_OK && e == cudaSuccess)
            e = cudaGraphInstantiate(&gg.graph, g, 0);
        if (g)
            cudaGraphDestroy(g);
        if (rc != OPO_OK || e != cudaSuccess) {
            cudaGetLastError();
            gg.graph = nullptr;
            return OPO_E_CUDA;
        }
    }
    for (int64_t i = 0; i < m && rc == OPO_OK; i++)
        rc = cuda_status(cudaGraphLaunch(gg.graph, s));
    if (rc == OPO_OK)
        rc = plain_batch_finalize(gg.d_calls, count, m, s);
    return rc;
}

} // namespace

int opo_batch_set_fields(opo_batch *b, const double *host, size_t count)
{
    if (!b || !host)
        return OPO_E_INVALID;
    size_t total = 0;
    for (const opo_ctx *c : b->ctxs)
        total += (size_t)c->F * c->n;
    if (count != total)
        return OPO_E_INVALID;
    DeviceGuard g(b->device);
    if (!g.ok)
        return OPO_E_CUDA;
    int rc = batch_staging(b, 2 * total);
    if (rc != OPO_OK)
        return rc;
    cudaStream_t s = b->stream;
    batch_fence(b, s, true);
    rc = batch_members(b, s);
    if (rc != OPO_OK)
        return rc;
    if (cudaMemcpyAsync(b->d_xfer, host, sizeof(double) * 2 * total, cudaMemcpyHostToDevice, s) !=
        cudaSuccess)
        return OPO_E_CUDA;
    k_batch_from_f64<<<xblocks((long long)total), 256, 0, s>>>(b->d_mem, (int)b->ctxs.size(),
                                                               b->d_xfer, (long long)total);
    if (cudaGetLastError() != cudaSuccess)
        return OPO_E_CUDA;
    batch_fence(b, s, false);
    // the host buffer is free to reuse when this returns
    return cudaStreamSynchronize(s) == cudaSuccess ? OPO_OK : OPO_E_CUDA;
}

int opo_batch_get_fields(opo_batch *b, int32_t field, int32_t which, double *host, size_t count)
{
    if (!b || !host || field < 0 || field > 2 || (which != OPO_INTRACAVITY && which != OPO_OUTPUT))
        return OPO_E_INVALID;
    size_t total = 0;
    for (const opo_ctx *c : b->ctxs)
        total += (size_t)c->n;
    if (count != total)
        return OPO_E_INVALID;
    DeviceGuard g(b->device);
    if (!g.ok)
        return OPO_E_CUDA;
    int rc = batch_staging(b, 2 * total);
    if (rc != OPO_OK)
        return rc;
    cudaStream_t s = b->stream;
    batch_fence(b, s, true);
    rc = batch_members(b, s);
    if (rc != OPO_OK)
        return rc;
    k_batch_to_f64<<<xblocks((long long)total), 256, 0, s>>>(b->d_mem, (int)b->ctxs.size(), field,
                                                             which, b->d_xfer, (long long)total);
    if (cudaGetLastError() != cudaSuccess)
        return OPO_E_CUDA;
    if (cudaMemcpyAsync(host, b->d_xfer, sizeof(double) * 2 * total, cudaMemcpyDeviceToHost, s) !=
        cudaSuccess)
        return OPO_E_CUDA;
    batch_fence(b, s, false);
    return batch_check_err(b);
}

int opo_batch_get_trace(opo_batch *b, double *host, int64_t rows)
{
    if (!b || !host || rows < 0)
        return OPO_E_INVALID;
    for (const opo_ctx *c : b->ctxs)
        if (rows > c->last_M)
            return OPO_E_INVALID;
    DeviceGuard g(b->device);
    if (!g.ok)
        return OPO_E_CUDA;
    const size_t per = 4 * (size_t)rows;
    int rc = batch_staging(b, per * b->ctxs.size());
    if (rc != OPO_OK)
        return rc;
    cudaStream_t s = b->stream;
    batch_fence(b, s, true);
    rc = batch_members(b, s);
    if (rc != OPO_OK)
        return rc;
    if (rows > 0) {
        k_batch_trace<<<xblocks((long long)per * (long long)b->ctxs.size()), 256, 0, s>>>(
            b->d_mem, (int)b->ctxs.size(), (int)rows, b->d_xfer);
        if (cudaGetLastError() != cudaSuccess)
            return OPO_E_CUDA;
    }
    if (rows > 0 && cudaMemcpyAsync(host, b->d_xfer, sizeof(double) * per * b->ctxs.size(),
                                    cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return OPO_E_CUDA;
    batch_fence(b, s, false);
    return batch_check_err(b);
}

int opo_batch_run(opo_batch *b, int64_t m)
{
    if (!b || m < 0)
        return OPO_E_INVALID;
    for (const opo_ctx *c : b->ctxs)
        if (c->d_hist && m > c->hist_cap)
            return OPO_E_INVALID;
    opo_ctx *c0 = b->ctxs[0];
    DeviceGuard g(c0->device);
    if (!g.ok)
        return OPO_E_CUDA;
    cudaStream_t s = c0->stream;
    const int count = (int)b->ctxs.size();
    for (const BatchGroup &gg : b->groups) {
        if (group_stale(gg, b->one_launch))
            return OPO_E_STATE;
        for (opo_ctx *c : gg.ctxs) {
            int rc = begin_call(c, m, gg.plain ? 1 : gg.cfg.cluster, false);
            if (rc != OPO_OK)
                return rc;
        }
    }
    for (int i = 0; i < count; i++) {
        opo_ctx *c = b->ctxs[i];
        if (c->stream != s) {
            cudaEventRecord(b->ev[i], c->stream);
            cudaStreamWaitEvent(s, b->ev[i], 0);
        }
    }
    int rc = OPO_OK;
    auto run_group = [&](BatchGroup &gg, cudaStream_t gs) {
        return gg.plain ? run_plain_group(b, gg, m, gs)
                        : fused_run(gg.ctxs.data(), (int)gg.ctxs.size(), gg.cfg, m, gs);
    };
    if (m > 0) {
        if (b->groups.size() == 1) {
            rc = run_group(b->groups[0], s);
        } else {
            cudaEventRecord(b->fork, s);
            for (BatchGroup &gg : b->groups) {
                if (rc != OPO_OK)
                    break;
                cudaStreamWaitEvent(gg.stream, b->fork, 0);
                rc = run_group(gg, gg.stream);
                cudaEventRecord(gg.done, gg.stream);
                cudaStreamWaitEvent(s, gg.done, 0);
            }
        }
    }
    for (const BatchGroup &gg : b->groups)
        for (opo_ctx *c : gg.ctxs) {
            c->rt += m;
            c->last_M = m;
            c->last_parts = gg.plain ? 1 : gg.cfg.cluster;
            c->last_path = gg.plain ? OPO_PATH_PLAIN : OPO_PATH_FUSED;
            c->last_cluster = gg.plain ? 0 : gg.cfg.cluster;
        }
    for (int i = 0; i < count; i++) {
        opo_ctx *c = b->ctxs[i];
        if (c->stream != s) {
            cudaEventRecord(b->ev[i], s);
            cudaStreamWaitEvent(c->stream, b->ev[i], 0);
        }
    }
    return rc;
}

int opo_batch_step_io(opo_batch *b, const double *host_in, double *host_out, int32_t field,
                      int64_t m)
{
    if (!b || m < 1 || field < 0)
        return OPO_E_INVALID;
    size_t n_in = 0, n_out = 0;
    for (const opo_ctx *c : b->ctxs) {
        if (field >= c->F || (c->d_hist && m > c->hist_cap))
            return OPO_E_INVALID;
        n_in += (size_t)c->F * c->n;
        n_out += (size_t)c->n;
    }
    const int count = (int)b->ctxs.size();
    const size_t in_doubles = 2 * n_in, out_doubles = 2 * n_out + 4 * (size_t)count;
    DeviceGuard g(b->device);
    if (!g.ok)
        return OPO_E_CUDA;
    // first use: the copy streams, events and staging slots
    if (!b->io_in) {
        bool ok = cudaStreamCreateWithFlags(&b->io_in, cudaStreamNonBlocking) == cudaSuccess &&
                  cudaStreamCreateWithFlags(&b->io_out, cudaStreamNonBlocking) == cudaSuccess;
        for (int k = 0; ok && k < 2; k++)
            ok = cudaEventCreateWithFlags(&b->ev_h2d[k], cudaEventDisableTiming) == cudaSuccess &&
                 cudaEventCreateWithFlags(&b->ev_used[k], cudaEventDisableTiming) == cudaSuccess &&
                 cudaEventCreateWithFlags(&b->ev_gath[k], cudaEventDisableTiming) == cudaSuccess &&
                 cudaEventCreateWithFlags(&b->ev_d2h[k], cudaEventDisableTiming) == cudaSuccess &&
                 cudaMalloc((void **)&b->d_in[k], sizeof(double) * in_doubles) == cudaSuccess &&
                 cudaMalloc((void **)&b->d_out[k], sizeof(double) * out_doubles) == cudaSuccess;
        if (!ok) {
            cudaGetLastError();
            return OPO_E_NOMEM;
        }
        for (int k = 0; k < 2; k++) { // nothing pending on either slot yet
            cudaEventRecord(b->ev_used[k], b->io_in);
            cudaEventRecord(b->ev_d2h[k], b->io_out);
        }
    }
    const int slot = b->io_slot;
    cudaStream_t s = b->stream;
    batch_fence(b, s, true);
    int rc = batch_members(b, s);
    if (rc != OPO_OK)
        return rc;
    if (host_in) {
        // the slot's previous input has been consumed two steps ago
        cudaStreamWaitEvent(b->io_in, b->ev_used[slot], 0);
        if (cudaMemcpyAsync(b->d_in[slot], host_in, sizeof(double) * in_doubles,
                            cudaMemcpyHostToDevice, b->io_in) != cudaSuccess)
            return OPO_E_CUDA;
        cudaEventRecord(b->ev_h2d[slot], b->io_in);
        cudaStreamWaitEvent(s, b->ev_h2d[slot], 0);
        k_batch_from_f64<<<xblocks((long long)n_in), 256, 0, s>>>(b->d_mem, count, b->d_in[slot],
                                                                  (long long)n_in);
        cudaEventRecord(b->ev_used[slot], s);
    }
    batch_fence(b, s, false);
    rc = opo_batch_run(b, m);
    if (rc != OPO_OK)
        return rc;
    if (host_out) {
        batch_fence(b, s, true);
        // the run may have moved the traces (they grow with m)
        rc = batch_members(b, s);
        if (rc != OPO_OK)
            return rc;
        // the slot's previous output has left for the host two steps ago
        cudaStreamWaitEvent(s, b->ev_d2h[slot], 0);
        k_batch_to_f64<<<xblocks((long long)n_out), 256, 0, s>>>(
            b->d_mem, count, field, OPO_OUTPUT, b->d_out[slot], (long long)n_out);
        // the last trace row of every member (the trace holds this call's m rows)
        k_batch_last_row<<<xblocks(4LL * count), 256, 0, s>>>(b->d_mem, count, (int)m,
                                                              b->d_out[slot] + 2 * n_out);
        cudaEventRecord(b->ev_gath[slot], s);
        batch_fence(b, s, false);
        cudaStreamWaitEvent(b->io_out, b->ev_gath[slot], 0);
        if (cudaMemcpyAsync(host_out, b->d_out[slot], sizeof(double) * out_doubles,
                            cudaMemcpyDeviceToHost, b->io_out) != cudaSuccess)
            return OPO_E_CUDA;
        cudaEventRecord(b->ev_d2h[slot], b->io_out);
    }
    if (cudaGetLastError() != cudaSuccess)
        return OPO_E_CUDA;
    b->io_slot = slot ^ 1;
    return OPO_OK;
}

int opo_batch_io_wait(opo_batch *b)
{
    if (!b)
        return OPO_E_INVALID;
    DeviceGuard g(b->device);
    if (!g.ok)
        return OPO_E_CUDA;
    for (cudaStream_t st : {b->io_in, b->io_out})
        if (st && cudaStreamSynchronize(st) != cudaSuccess)
            return OPO_E_CUDA;
    return batch_check_err(b);
}

int opo_batch_set_one_launch(opo_batch *b, int32_t on)
{
    if (!b || (on != 0 && on != 1))
        return OPO_E_INVALID;
    DeviceGuard g(b->device);
    if (!g.ok)
        return OPO_E_CUDA;
    cudaDeviceSynchronize(); // the groups' streams and graphs may be in use
    // the fused members, in batch order
    std::vector<opo_ctx *> fused;
    std::vector<BatchGroup> plain;
    for (BatchGroup &gg : b->groups) {
        if (gg.plain) {
            plain.push_back(gg);
            gg.d_insts = nullptr; // moved
            gg.d_calls = nullptr;
            gg.graph = nullptr;
        }
    }
    for (opo_ctx *c : b->ctxs)
        for (const BatchGroup &gg : b->groups)
            if (!gg.plain && std::find(gg.ctxs.begin(), gg.ctxs.end(), c) != gg.ctxs.end())
                fused.push_back(c);
    std::vector<BatchGroup> groups;
    if (!fused.empty()) {
        if (on) {
            // one launch: a configuration holding every fused member (the
            // generic kernel when sizes or field counts differ)
            int fmin = 3, fmax = 2, nmin = 1 << 17, nmax = 16, rtpl = 0;
            bool kerr = false, dk = false;
            for (const opo_ctx *c : fused) {
                fmin = std::min(fmin, c->F);
                fmax = std::max(fmax, c->F);
                nmin = std::min(nmin, c->n);
                nmax = std::max(nmax, c->n);
                rtpl = std::max(rtpl, c->rtpl_req);
                kerr = kerr || c->kerr_any;
                dk = dk || c->dk_any;
            }
            BatchGroup gg;
            gg.ctxs = fused;
            const int nl = kerr ? kNlKerr : (dk ? kNlChi2 : kNlChi2NoDk);
            if (!fused_config(fused[0]->csz, fmin, fmax, nmin, nmax, 0, rtpl, 0, nl, &gg.cfg))
                return OPO_E_UNSUPPORTED;
            groups.push_back(gg);
        } else {
            // back to one launch per size class: rebuild the batch's groups
            opo_batch *t = nullptr;
            int rc = opo_batch_create(&t, fused.data(), (int)fused.size(), 0, 0);
            if (rc != OPO_OK)
                return rc;
            for (BatchGroup &gg : t->groups)
                if (!gg.plain) {
                    BatchGroup x;
                    x.ctxs = gg.ctxs;
                    x.cfg = gg.cfg;
                    groups.push_back(x);
                }
            opo_batch_destroy(t);
        }
    }
    for (BatchGroup &gg : b->groups) {
        if (gg.stream)
            cudaStreamDestroy(gg.stream);
        if (gg.done)
            cudaEventDestroy(gg.done);
        if (gg.graph)
            cudaGraphExecDestroy(gg.graph);
        if (gg.d_insts)
            cudaFree(gg.d_insts);
        if (gg.d_calls)
            cudaFree(gg.d_calls);
    }
    for (BatchGroup &gg : plain)
        groups.push_back(gg);
    b->groups = groups;
    int rc = OPO_OK;
    if (b->groups.size() > 1)
        for (BatchGroup &gg : b->groups) {
            gg.stream = nullptr;
            gg.done = nullptr;
            if (rc == OPO_OK)
                rc = cuda_status(cudaStreamCreateWithFlags(&gg.stream, cudaStreamNonBlocking));
            if (rc == OPO_OK)
                rc = cuda_status(cudaEventCreateWithFlags(&gg.done, cudaEventDisableTiming));
        }
    else
        for (BatchGroup &gg : b->groups) {
            gg.stream = nullptr;
            gg.done = nullptr;
        }
    b->one_launch = on != 0;
    return rc;
}

int opo_batch_destroy(opo_batch *b)
{
    if (!b)
        return OPO_OK;
    DeviceGuard g(b->device);
    // the batch's events may still be pending on the device
    cudaDeviceSynchronize();
    batch_free(b);
    return OPO_OK;
}

} // extern "C"
