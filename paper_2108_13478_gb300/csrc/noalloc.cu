// Spectral bounds of S^-1 F with no device allocation at all.
//
// Some callers cannot call cudaMalloc: code running inside another
// framework's memory pool with allocation disabled, a captured or
// pre-planned execution where every buffer must already exist, or an
// embedded caller that only owns a fixed set of buffers.  This entry point
// gives them the Lanczos bounds of S^-1 F (the same computation that
// dft_density_matrix runs before the Chebyshev expansion) using a
// file-scope device array as its scratch instead of any allocation.
//
// The scratch holds two K x K FP64 matrices, four Lanczos vectors and the
// tridiagonal coefficients for K <= DFT_STATIC_MAX_K (768): about 9.5 MB
// that every GPU which loads the library keeps until the process exits.
#include "dft_internal.cuh"

#include <mutex>

namespace dft {
namespace {

constexpr int MAX_K = 768;
constexpr size_t SCRATCH_DOUBLES = 2ull * MAX_K * MAX_K + 4ull * MAX_K + SCAL_COUNT;

static __device__ __align__(256) double g_static_scratch[SCRATCH_DOUBLES];

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
double* g_addr[MAX_DEVICES] = {};

// device address of the static array on the current device, looked up once
// per device (host code only sees a host-side stand-in under its name)
double* scratch_address() {
    int dev = 0;
    DFT_CUDA_CHECK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= MAX_DEVICES) throw Error(DFT_EINVAL, "device index beyond the static scratch table");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || !p)
            throw Error(DFT_ECUDA, std::string("cudaGetSymbolAddress(static scratch): ") + cudaGetErrorString(e));
        g_addr[dev] = static_cast<double*>(p);
    }
    return g_addr[dev];
}

}  // namespace
}  // namespace dft

using namespace dft;

extern "C" dft_status dft_spectral_bounds_static(dft_ctx* ctx, const double* F, double* bounds, void* stream) {
    if (!ctx) return DFT_EINVAL;
    Ctx& c = *reinterpret_cast<Ctx*>(ctx);
    try {
        if (c.K == 0 || !F || !bounds) throw Error(DFT_EINVAL, "null argument");
        require_aligned16({F});
        if (c.K > MAX_K)
            throw Error(DFT_EINVAL, "K = " + std::to_string(c.K) + " exceeds the static scratch limit of " +
                                        std::to_string(MAX_K) + " basis functions");
        if (!c.have_chol) throw Error(DFT_EINVAL, "call dft_overlap_kinetic first");
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        double* base = scratch_address();
        const int K = c.K;
        double* tmp = base;
        double* Ft = base + (size_t)MAX_K * MAX_K;
        double* vec = base + 2ull * MAX_K * MAX_K;
        double* scal = vec + 4ull * MAX_K;
        if (c.p.e_max > c.p.e_min) {
            // fixed bounds in the parameters: dft_density_matrix takes them as
            // they are, without Lanczos
            bounds[0] = c.p.e_min;
            bounds[1] = c.p.e_max;
            c.err.clear();
            return DFT_OK;
        }
        // the scalar block starts from zero on every call (the array keeps the
        // previous call's contents)
        DFT_CUDA_CHECK(cudaMemsetAsync(scal, 0, sizeof(double) * SCAL_COUNT, s));
        congruence_lower(K, c.d_Linv, F, tmp, Ft, s);
        lanczos_bounds_at(K, Ft, c.p.lanczos_steps > 0 ? c.p.lanczos_steps : 64, c.p.seed, vec, scal, s);
        DFT_CUDA_CHECK(cudaMemcpyAsync(bounds, scal + SCAL_EMIN, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
        DFT_CUDA_CHECK(cudaStreamSynchronize(s));
        c.err.clear();
        return DFT_OK;
    } catch (const Error& e) {
        c.err = e.msg;
        return e.code;
    } catch (...) {
        c.err = "internal error";
        return DFT_EINTERNAL;
    }
}
