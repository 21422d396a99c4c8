// opo_internal.h -- host-side state of a libopo context and the launchers
// that the C-ABI file (opo_abi.cu) calls in the kernel files.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/opo.h"
#include "opo_common.cuh"

namespace opo {

constexpr double kPi = 3.141592653589793238462643383279502884;
constexpr double kEps0 = 8.8541878128e-12; // vacuum permittivity [F/m]
constexpr double kC0 = 299792458.0;        // speed of light [m/s]
constexpr int kNslot = 5;                  // raw observable sums per round trip

// Device control block read by every per-round-trip kernel, so that one
// captured graph serves every round trip of a call.
struct DevCtl {
    int64_t rt0;      // absolute round-trip index of slot 0 of the current call
    int64_t slot;     // round trip within the current call
    double *obs;      // raw sums [slot][parts][kNslot]
    int32_t parts;    // partial sums per slot (CTAs per instance; 1 on the plain path)
    int32_t err;      // sticky error word: bit 0 a non-finite field; bit 1 is
                      // reserved for a bounded device wait that gave up (the
                      // kernels hold no such wait: clusters meet only at
                      // hardware cluster barriers)
};

// Scalars of one instance derived once on the host from crystal and cavity.
struct Derived {
    double kappa[3];     // 2 pi d_eff / (n lambda)
    double dz, h;        // step and RK4 half step
    double bc_re[3], bc_im[3]; // sqrt(R) e^{i delta} for resonant fields, 1 otherwise
    double outscale[3];  // sqrt(1 - R) for resonant fields, 1 otherwise
    double pscale[3];    // n eps0 c / 2 * pi w0^2
    bool use_dk;
    bool eom;
    bool kerr;             // chi(3) terms on
    double kerr_g[9];      // G_xy of the Kerr terms, row-major
    NsPump ns;           // ns-pulsed pump parameters (ns.on = 0: pump table)
};

constexpr int kMaxCry = OPO_MAX_CRYSTALS;

// Device-side description of one crystal of an instance's round trip.
struct CryDesc {
    const void *disp;   // F*N dispersion factors / N, natural order
    const void *disp_t; // the same, row-major over N = P Q
    const void *ekz;    // 4 nz + 1 factors e^{i dk q dz/4}
    double kappa[3], h; // 2 pi d_eff / (n lambda); RK4 half step dz/2
    int nz, use_dk, kerr;
    double kerr_g[9];   // Kerr coefficients G_xy, row-major
    float kf[13];       // kappa[0..2], h, kerr_g[0..8] rounded to float (the
                        // constants of the FP32 kernels, converted on the host)
};

// Tables of a crystal after the first (the first one's live in the
// context's d_disp, d_disp_t and d_ekz).
struct CrystalState {
    void *disp = nullptr, *disp_t = nullptr, *ekz = nullptr;
    int ekz_cap = 0;
};

// Nonlinear-step variants of the size-specialised fused kernel, each its own
// instantiation: chi(2) with the phase-mismatch factors switched by a runtime
// flag per crystal; chi(2) plus the Kerr terms; chi(2) where dk = 0 in every
// crystal (no phase factors at all: the RK4 step without its predicated
// products).
constexpr int kNlChi2 = 0, kNlKerr = 1, kNlChi2NoDk = 2;

// Cavity elements of the plain path's time-domain kernel: mirror
// sqrt(R) e^{i delta} and the EOM, on resonant fields.
struct PlainCav {
    double bc_re[3], bc_im[3];
    double eom_beta, eom_f, t_rt, dt;
    unsigned resmask;
    int eom;
};

// One member of a batched plain-path launch (a device array of these, one per
// instance; the batch kernels take instance blockIdx.z).  The same kernels'
// bodies run a lone context, so a member advances exactly as it would alone.
struct PlainInst {
    void *fields, *out, *scratch, *hist;
    const void *pump, *gdd, *tw;
    const CryDesc *cry;   // the instance's crystals (device copy)
    DevCtl *ctl;
    NsPump ns;
    PlainCav cav;
    double outscale[3];   // sqrt(1 - R) on resonant fields, else 1
    int spec_all;         // the cavity visit transforms every field (GDD or
                          // delay on a resonant field), else a signal copy
};

// Per-call values of a batch member: start of the call (round-trip counter,
// observable storage) and the trace rows it finalizes.
struct PlainCall {
    DevCtl *ctl;
    double *obs, *trace;
    int64_t rt0;
    double outscale2[3], pscale[3];
    double inv_n, t_window;
    int F;
};

struct FusedCfg {
    int kernel = 1;      // 1: generic, 2: size-specialised, 3: size-specialised in place,
                         // 4: in place with the exchange through global memory
    int nl = 0;          // kNl* variant (kernels 2, 3 instantiate each)
    int cluster;         // CTAs per instance
    int threads;         // threads per CTA
    int rt_per_launch;   // round trips per launch
    bool disp_in_smem;   // dispersion factors resident in shared memory
    size_t smem;         // dynamic shared memory per CTA
};

} // namespace opo

struct opo_ctx {
    opo_grid grid;
    opo_crystal crystal;                  // the first crystal (== cry[0])
    opo_crystal cry[OPO_MAX_CRYSTALS];    // every crystal of the round trip
    int ncry = 1;
    opo::CrystalState xs[OPO_MAX_CRYSTALS]; // tables of crystals 1..ncry-1
    opo::CryDesc h_cry[OPO_MAX_CRYSTALS]; // host copy of the descriptors
    opo::CryDesc *d_cry = nullptr;        // their device copy (kMaxCry entries)
    bool kerr_any = false;                // some crystal has Kerr terms
    bool dk_any = false;                  // some crystal has dk != 0
    opo_cavity cavity;
    bool have_crystal = false, have_cavity = false;
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaStream_t capture_stream = nullptr;
    int n = 0, logn = 0, F = 0, prec = 0;
    size_t csz = 0; // bytes per complex element
    // device memory (complex arrays in the context's precision)
    void *d_fields = nullptr;  // F*N intracavity state
    void *d_out = nullptr;     // F*N output-coupled fields of the last round trip
    void *d_scratch = nullptr; // F*N FFT intermediate of the plain path; also the
                               // forward exchange buffer of the fused form that
                               // exchanges through global memory
    void *d_xg = nullptr;      // F*N inverse exchange buffer of that form (the
                               // sizes that need it only)
    void *d_pump = nullptr;    // N input pump
    void *d_disp = nullptr;    // F*N dispersion factors / N, natural order
    void *d_gdd = nullptr;     // F*N cavity spectral factors / N, natural order
    // the same two tables row-major over N = P Q, P = 2^(logn/2): entry
    // [x][k1][k2] holds bin k = k1 + k2 P (the order in which the in-place
    // fused kernel visits a row spectrum, so that its loads coalesce)
    void *d_disp_t = nullptr;
    void *d_gdd_t = nullptr;
    void *d_tw = nullptr;      // N twiddles W_N^j = e^{-2 pi i j/N}
    void *d_ekz = nullptr;     // 4 nz + 1 factors e^{i dk q dz/4}
    int ekz_cap = 0;
    double *d_pump_user = nullptr; // staging for OPO_PUMP_USER (FP64)
    double *d_stage = nullptr;     // 2N doubles: host <-> device field staging
    void *d_hist = nullptr;    // output history: hist_cap rows of F*N (optional)
    int64_t hist_cap = 0;
    double *d_obs = nullptr;   // raw observable sums
    double *d_trace = nullptr; // rows {P_p, P_s, P_i, nu_c}
    int64_t obs_cap = 0;       // capacity in round trips (times parts)
    int obs_parts_cap = 0;
    opo::DevCtl *d_ctl = nullptr;
    double *h_pinned = nullptr; // small pinned staging
    int64_t rt = 0;            // round-trip counter m
    int64_t last_M = 0;        // round trips in the last call
    int last_parts = 1;
    opo::Derived dv{};
    int path_req = OPO_PATH_AUTO, cluster_req = 0, rtpl_req = 0, threads_req = 0;
    int last_path = OPO_PATH_PLAIN, last_cluster = 0;
    cudaGraphExec_t graph = nullptr;
    bool graph_valid = false;
    uint64_t gen = 0;          // bumped whenever crystals, cavity or history change
};

namespace opo {

// opo_abi.cu: argument checks shared by the context calls, opo_validate
// and the allocation-free pass (no device access)
bool valid_grid_shape(const opo_grid *g);
bool valid_crystal_for(int F, const opo_crystal *k);
bool valid_crystals_for(int F, const opo_crystal *list, int count);
bool valid_cavity_for(int F, int n, const opo_cavity *v);

// opo_setup.cu
int setup_twiddles(opo_ctx *c);
// tables of every crystal and the device copy of their descriptors
int setup_crystal_tables(opo_ctx *c);
int setup_cavity_tables(opo_ctx *c);
int finalize_trace(opo_ctx *c, int64_t M, int parts);
// twiddles, dispersion factors and e^{i dk q dz/4} into caller-given buffers
int setup_pass_tables(void *tw, void *disp, void *ekz, int n, int F, bool dbl,
                      const opo_crystal &k, double t_window, cudaStream_t s);

// opo_plain.cu
void plain_prepare(opo_ctx *c);
int plain_enqueue_roundtrip(opo_ctx *c, cudaStream_t s);
// the batched plain path: members' descriptors, one captured round trip of
// every member (c0 gives N, F, precision and the crystals' step counts, the
// same in every member), and the per-call start and trace of every member
void plain_fill_inst(PlainInst &p, const opo_ctx *c);
void plain_fill_call(PlainCall &p, const opo_ctx *c);
int plain_batch_enqueue_roundtrip(const opo_ctx *c0, const PlainInst *d_insts, int count,
                                  cudaStream_t s);
int plain_batch_begin(const PlainCall *d_calls, int count, cudaStream_t s);
int plain_batch_finalize(const PlainCall *d_calls, int count, int64_t M, cudaStream_t s);
// one crystal pass of the plain kernels on caller-given buffers
int plain_pass_raw(void *fields, void *scratch, const void *tw, const void *disp, const void *ekz,
                   int n, int F, int nz, const double kappa[3], double h, bool use_dk,
                   const double *kerr_g, bool dbl, cudaStream_t st);

// opo_setup.cu: coefficients G_xy (row-major 3 x 3) of the Kerr terms of a
// crystal; false (all zero) when its n2 is 0.
bool kerr_coefficients(const opo_crystal &k, int F, double g[9]);

// the size-specialised kernel variant an instance needs (kNl*)
inline int nl_variant(const opo_ctx *c)
{
    return c->kerr_any ? kNlKerr : (c->dk_any ? kNlChi2 : kNlChi2NoDk);
}

// opo_fused.cu: a cluster configuration able to hold instances with up to
// fmax fields and nmin..nmax points and nonlinear-step variant nl (false if
// none fits or can launch).
bool fused_config(size_t csz, int fmin, int fmax, int nmin, int nmax, int cluster_req,
                  int rtpl_req, int threads_req, int nl, FusedCfg *out);
int fused_max_active(bool dbl, int F, int n, const FusedCfg &cfg);
int fused_run(opo_ctx *const *ctxs, int count, const FusedCfg &cfg, int64_t m, cudaStream_t s);

} // namespace opo
