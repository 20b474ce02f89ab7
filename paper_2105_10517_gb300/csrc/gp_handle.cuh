// gp_handle.cuh -- the device state behind a gp_handle and the runtime helpers
// shared by the C-ABI translation units (gp_capi.cu, gp_batch.cu).
#pragma once
#include <nvtx3/nvToolsExt.h>

#include "gp_internal.cuh"

namespace gpspin {

constexpr int kNormBlocksMax = 16384;

// NVTX range over a library call (visible to ncu --nvtx and other profilers;
// a no-op when no tool is attached).
struct TraceRange {
    explicit TraceRange(const char* name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange&) = delete;
    TraceRange& operator=(const TraceRange&) = delete;
};

// Coefficient tables and tilings of one mode (imaginary or real time).
struct CoefSet {
    bool valid = false;
    gp_params key{};
    LineCoef* cx = nullptr;   // [ny][3] x-pass lines (rows), FP64
    LineCoef* cy = nullptr;   // [nx][3] y-pass lines (columns), FP64
    double2* ex = nullptr;    // [nx]
    double2* ey = nullptr;    // [ny]
    LineCoefF* fx = nullptr;  // complex64 copies (FP32-storage handles only)
    LineCoefF* fy = nullptr;
    float2* fex = nullptr;
    float2* fey = nullptr;
    LineTiling tx{}, ty{}, ftx{}, fty{};  // single-instance launches (may span 2-CTA clusters)
    LineTiling ux{}, uy{}, fux{}, fuy{};  // unsplit, for batched launches
    // second-order splitting (complex128): x-pass tables and trap factors of dt/2
    bool half_valid = false;
    LineCoef* cxh = nullptr;
    double2* exh = nullptr;
    double2* eyh = nullptr;
};

}  // namespace gpspin

struct gp_handle {
    gp_params p{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int device = 0;
    int active = GP_FP64;      // precision of the propagated copy
    double2* psi = nullptr;    // [3][ny][nx] complex128 state (authoritative when active == GP_FP64)
    double2* work = nullptr;   // [3][nx][ny] transposed intermediate / staging
    float2* psi32 = nullptr;   // complex64 state (authoritative when active == GP_FP32_MIXED)
    float2* work32 = nullptr;
    double* partials = nullptr;
    double* obs_part = nullptr;
    double* scal = nullptr;    // [0] pending normalisation, [1] last norm, [2] the constant 1,
                               // [3..5] per-component factors of the constrained normalisation
    double* obs_out = nullptr; // [8]
    int* flag = nullptr;       // bit0 coefficient convergence, bit1 norm, bit2 observables, bit3 copy timeout
    gpspin::CoefSet coef[2];   // per mode
    cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};  // gp_profile_step
    cudaGraphExec_t graph[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};  // [precision][mode]
    bool scale_pending = false;
    long long steps = 0;
    int mcon = 0;              // imaginary time keeps N = 1 and N+ - N- = m_target
    double m_target = 0.0;
    int split = 0;             // GP_SPLIT_LIE or GP_SPLIT_STRANG
    int debug = 0;             // GP_DEBUG_* flags
};

namespace gpspin {

// Runtime helpers (gp_capi.cu).
// Every device allocation of the library goes through dev_alloc, which honours
// the failure injection of gp_inject_alloc_failure.
int dev_alloc(void** p, size_t bytes);
template <typename T>
bool dalloc(T** p, size_t bytes)
{
    return dev_alloc(reinterpret_cast<void**>(p), bytes) == GP_OK;
}
int ensure_coef(gp_handle* h, int mode);
PassArgs pass_args(gp_handle* h, const CoefSet& cs, int dir);
PassArgsF pass_args_f32(gp_handle* h, const CoefSet& cs, int dir);
size_t n_elems(const gp_handle* h);
double cell(const gp_handle* h);
int y_blocks(const LineTiling& t);
int flush_scale(gp_handle* h);
// Bytes of device memory gp_create allocates for these parameters, plus the
// coefficient tables of one mode.
size_t handle_bytes(const gp_params& p);

}  // namespace gpspin
