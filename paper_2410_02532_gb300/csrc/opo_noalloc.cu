// opo_noalloc.cu -- opo_crystal_pass_noalloc: one crystal pass of the plain
// kernels on caller-owned device fields, for callers that cannot allocate
// device memory (for example code running inside another framework's memory
// pool, or a process whose allocator is locked down).  Its scratch (FFT
// intermediate, twiddles, dispersion factors, e^{i dk z} factors) lives in
// one file-scope device array, so the call itself allocates nothing.
#include <cmath>

#include "opo_common.cuh"
#include "opo_internal.h"

namespace {

constexpr size_t kScratchBytes = size_t(4) << 20; // 4 MiB
constexpr int kMaxDevices = 64;

// Shared by every call on a device; every GPU that loads the library holds it
// until the process exits.
static __device__ __align__(256) unsigned char opo_noalloc_scratch[kScratchBytes];

// Device address of the array on the current device, looked up on every
// call (a lookup allocates nothing; a cached address would go stale when
// the module is loaded again after a device reset).
int scratch_for(void **out)
{
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, opo_noalloc_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return OPO_E_CUDA;
    }
    *out = p;
    return OPO_OK;
}

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

} // namespace

extern "C" OPO_API int opo_crystal_pass_noalloc(const opo_grid *grid, const opo_crystal *k,
                                                void *fields, void *stream)
{
    if (!grid || !k || !fields)
        return OPO_E_INVALID;
    // the checks of opo_create and opo_set_crystal
    if (!opo::valid_grid_shape(grid) || !opo::valid_crystal_for(grid->nfields, k))
        return OPO_E_INVALID;
    const int n = grid->n;
    const int F = grid->nfields;
    const bool dbl = grid->precision == OPO_FP64;
    const size_t csz = dbl ? sizeof(double2) : sizeof(float2);
    // scratch layout: twiddles N | FFT intermediate F*N | dispersion F*N | ekz 4 nz + 1
    const size_t b_tw = align256(csz * n);
    const size_t b_scr = align256(csz * (size_t)F * n);
    const size_t b_disp = align256(csz * (size_t)F * n);
    const size_t b_ekz = align256(csz * (size_t)(4 * k->nz + 1));
    if (b_tw + b_scr + b_disp + b_ekz > kScratchBytes)
        return OPO_E_INVALID; // beyond the fixed scratch: use the context API
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
        cudaGetLastError();
        return OPO_E_CUDA;
    }
    if (grid->device < 0 || grid->device >= ndev || grid->device >= kMaxDevices)
        return OPO_E_INVALID;
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess)
        prev = -1;
    if (cudaSetDevice(grid->device) != cudaSuccess)
        return OPO_E_CUDA;
    void *base = nullptr;
    int rc = scratch_for(&base);
    if (rc == OPO_OK) {
        cudaStream_t s = (cudaStream_t)stream;
        char *b = (char *)base;
        void *tw = b, *scr = b + b_tw, *disp = b + b_tw + b_scr, *ekz = b + b_tw + b_scr + b_disp;
        rc = opo::setup_pass_tables(tw, disp, ekz, n, F, dbl, *k, grid->t_window_s, s);
        if (rc == OPO_OK) {
            double kappa[3] = {0.0, 0.0, 0.0};
            for (int x = 0; x < F; x++)
                kappa[x] = 2.0 * opo::kPi * k->deff_mpv / (k->n[x] * k->lambda_m[x]);
            const double h = 0.5 * k->length_m / (double)k->nz;
            double kg[9];
            const bool kerr = opo::kerr_coefficients(*k, F, kg);
            rc = opo::plain_pass_raw(fields, scr, tw, disp, ekz, n, F, k->nz, kappa, h,
                                     k->dk_per_m != 0.0, kerr ? kg : nullptr, dbl, s);
        }
    }
    if (prev >= 0)
        cudaSetDevice(prev);
    return rc;
}
