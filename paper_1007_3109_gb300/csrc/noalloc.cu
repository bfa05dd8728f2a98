// Allocation-free variant of the fused step (declared in include/lb_rd.h as
// lb_rd_step_noalloc).  Some callers cannot call cudaMalloc: a real-time loop
// whose device memory was all reserved at start-up, or a plugin that may only
// use the buffers its host application hands it.  This entry point runs one
// time step between two caller-owned state buffers and reduces the FP64 mass,
// and it takes the reduction's scratch (per-block partial sums plus the
// arrival counter of the last-block finalisation) from a fixed array in this
// file instead of allocating it.
#include <cuda_runtime.h>

#include <map>
#include <mutex>
#include <string>

#include "lb_rd.h"
#include "lbrd_kernels.h"

namespace lbrd {
int report_error(int code, const std::string &msg);
}

// Partial sums for up to kNoAllocSlots (tile, species) pairs: 512 KiB, then
// one 256-byte slot that holds the arrival counter.  Every GPU that loads the
// library holds this array until the process exits.
constexpr int64_t kNoAllocSlots = 65536;
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocSlots + 32];

namespace {

std::mutex g_mu;
std::map<int, double *> g_scratch_addr;  // device ordinal -> device address of g_noalloc_scratch

// Device address of the scratch array on the current device.  In host code
// the array's name is only a host-side stand-in, so the address is looked up
// once per device (with that device current, in the runtime's primary
// context) and cached by device ordinal.
int scratch_on_current_device(double **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return lbrd::report_error(LB_RD_ECUDA, std::string("lb_rd_step_noalloc: no CUDA device: ") + cudaGetErrorString(e));
    std::lock_guard<std::mutex> lock(g_mu);
    auto it = g_scratch_addr.find(dev);
    if (it != g_scratch_addr.end()) {
        *out = it->second;
        return LB_RD_OK;
    }
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr)
        return lbrd::report_error(LB_RD_ECUDA, std::string("lb_rd_step_noalloc: cudaGetSymbolAddress failed: ") +
                                                   cudaGetErrorString(e));
    g_scratch_addr[dev] = static_cast<double *>(p);
    *out = static_cast<double *>(p);
    return LB_RD_OK;
}

}  // namespace

extern "C" int lb_rd_step_noalloc(const lb_rd_config *cfg, const void *state_in, void *state_out, double *mass_out) {
    int rc = lb_rd_check_config(cfg, nullptr);
    if (rc) return rc;
    if (!state_in || !state_out || !mass_out)
        return lbrd::report_error(LB_RD_EINVAL, "lb_rd_step_noalloc: state_in, state_out and mass_out must be device pointers");
    if (state_in == state_out)
        return lbrd::report_error(LB_RD_EINVAL, "lb_rd_step_noalloc: state_in and state_out must be different buffers");
    if (cfg->nspecies > 2 || cfg->reaction.kind == LB_RD_REACTION_MASS_ACTION || cfg->streaming != 0)
        return lbrd::report_error(LB_RD_EINVAL,
                                  "lb_rd_step_noalloc: at most two species, no mass-action network, two state buffers");
    const int Q = cfg->lattice == LB_RD_D2Q9 ? 9 : 5;
    const int S = cfg->nspecies;
    const int prec = cfg->precision;
    const bool half = prec == LB_RD_FP32_BF16DEV || prec == LB_RD_FP32_FP16DEV;
    if (half && cfg->nx % 4 != 0)
        return lbrd::report_error(LB_RD_EINVAL, "lb_rd_step_noalloc: 16-bit deviation storage needs nx to be a multiple of 4");
    const int64_t ntiles = prec == LB_RD_FP64 ? lbrd::step_tiles_f64(cfg->nx, cfg->ny)
                           : prec == LB_RD_FP32 ? lbrd::step_tiles_f32(cfg->nx, cfg->ny)
                                                : lbrd::step_tiles_half(cfg->nx, cfg->ny);
    if (ntiles * S > kNoAllocSlots)
        return lbrd::report_error(
            LB_RD_EINVAL, "lb_rd_step_noalloc: grid too large for the static scratch: " + std::to_string(ntiles) +
                              " tiles x " + std::to_string(S) + " species need " + std::to_string(ntiles * S) +
                              " partial sums, the limit is " + std::to_string(kNoAllocSlots));
    double *scratch = nullptr;
    rc = scratch_on_current_device(&scratch);
    if (rc) return rc;

    lbrd::StepArgs a{};
    a.src = state_in;
    a.dst = state_out;
    a.nx = cfg->nx;
    a.ny = cfg->ny;
    a.pitch = lbrd::state_pitch(cfg->nx);  // the handles' layout (lb_rd_save payload)
    a.plane = cfg->ny * a.pitch;
    lbrd::fill_reaction(*cfg, a.omega, &a.rkind, &a.kappa, &a.F, &a.k, &a.net);
    a.rho_out = nullptr;
    a.partials = scratch;
    a.counter = reinterpret_cast<unsigned int *>(scratch + kNoAllocSlots);
    a.mass_out = mass_out;
    cudaStream_t st = static_cast<cudaStream_t>(cfg->stream);
    // The counter must start at zero; the array keeps whatever the last call left.
    cudaError_t e = cudaMemsetAsync(a.counter, 0, sizeof(unsigned int), st);
    if (e == cudaSuccess) {
        if (prec == LB_RD_FP64) e = lbrd::launch_step_f64_per_tile(Q, S, a, st);
        else if (prec == LB_RD_FP32) e = lbrd::launch_step_f32_per_tile(Q, S, a, st);
        else e = lbrd::launch_step_half_per_tile(Q, S, prec == LB_RD_FP32_FP16DEV, a, st);
    }
    if (e != cudaSuccess)
        return lbrd::report_error(LB_RD_ECUDA, std::string("lb_rd_step_noalloc: ") + cudaGetErrorName(e) + " (" +
                                                   cudaGetErrorString(e) + ")");
    return LB_RD_OK;
}
