// gd_noalloc.cu -- gd_solve_noalloc: the Newton-system Krylov solve for callers
// that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: an application that hands the whole device
// to its own memory pool (every byte belongs to the pool, so an allocation from
// outside it fails or breaks the pool's accounting), or an embedding runtime that
// forbids allocation once it has started (allocation can fail and synchronises the
// device, which such runtimes keep out of their steady state).  For them this
// entry point takes the CSR system and the vectors from the caller and keeps all
// of its work space (the nine BiCGStab vectors, the node-block inverses, the
// reduction partials and the result words) in one file-scope device array of
// fixed size.  Every GPU that loads the library holds that array until the
// process exits.  The call reads its iteration count and residual back to host
// memory and synchronises the caller's stream before it returns.
//
// The array is a device symbol: in host code its name is only a stand-in, so
// its device address is looked up once per device with cudaGetSymbolAddress
// (with that device current) and that address is what the kernels receive.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "gd_internal.cuh"

namespace {

constexpr int64_t kMaxDofs = GD_NOALLOC_MAX_DOFS;
constexpr int kMaxBlocks = 4096;                      // cooperative grid cap (reduction partial slots)
constexpr size_t kVec = (size_t)kMaxDofs;
// 9 Krylov vectors, node-block inverses (n_nodes * ndof^2 <= 4 * n_dofs), partials, result words
constexpr size_t kScratchDoubles = 9 * kVec + 4 * kVec + 8 * (size_t)kMaxBlocks + 8;

static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double *g_addr[kMaxDevices] = {};

}  // namespace

extern "C" gd_status gd_solve_noalloc(int32_t ndof, int64_t n_nodes, const int32_t *rowptr, const int32_t *colidx,
                                      const double *vals, const uint8_t *fixed, const double *b, double *x,
                                      double rtol, int32_t max_it, void *stream, int32_t *iterations,
                                      double *rel_residual)
{
    if (ndof != 3 && ndof != 4) return gd::set_error(GD_ERR_ARG, "gd_solve_noalloc: ndof must be 3 or 4");
    if (n_nodes <= 0 || !rowptr || !colidx || !vals || !fixed || !b || !x)
        return gd::set_error(GD_ERR_ARG, "gd_solve_noalloc: empty system or null pointer");
    if (n_nodes * ndof > kMaxDofs)
        return gd::set_error(GD_ERR_ARG, "gd_solve_noalloc: " + std::to_string(n_nodes * ndof) +
                                             " dofs exceed the fixed work space of " + std::to_string(kMaxDofs) +
                                             " dofs (use gd_solve)");
    if (!(rtol > 0.0) || max_it < 1) return gd::set_error(GD_ERR_ARG, "gd_solve_noalloc: rtol/max_it");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return gd::set_error(GD_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return gd::set_error(GD_ERR_ARG, "gd_solve_noalloc: device index too large");
    double *base = nullptr;
    {
        // one-time set-up per device, with that device current
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_addr[dev]) {
            e = cudaGetSymbolAddress((void **)&g_addr[dev], g_noalloc_scratch);
            if (e != cudaSuccess) {
                g_addr[dev] = nullptr;
                return gd::set_error(GD_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            }
        }
        base = g_addr[dev];
    }
    int num_sms = 0;
    e = cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return gd::set_error(GD_ERR_CUDA, std::string("cudaDeviceGetAttribute: ") + cudaGetErrorString(e));
    const int64_t n = n_nodes * ndof;
    gd::KrylovCtx kc;
    kc.n_nodes = n_nodes;
    kc.ndof = ndof;
    kc.rowptr = rowptr;
    kc.colidx = colidx;
    kc.fixed = fixed;
    for (int k = 0; k < 9; ++k) kc.work[k] = base + (size_t)k * n;
    kc.work_x = nullptr;
    kc.binv = base + 9 * kVec;
    kc.red = base + 13 * kVec;
    kc.out = kc.red + 8 * (size_t)kMaxBlocks;
    kc.stream = (cudaStream_t)stream;
    kc.num_sms = num_sms;
    kc.blocks = gd::krylov_blocks(ndof, false, num_sms);
    if (kc.blocks > kMaxBlocks) kc.blocks = kMaxBlocks;
    if (kc.blocks < 1) return gd::set_error(GD_ERR_CUDA, "gd_solve_noalloc: no cooperative grid fits");
    // nothing left in the array by an earlier call reaches this one: krylov_solve
    // zeroes the grid-wide accumulator words (atomic sums) with a memset before its
    // launch, and every work vector, block partial and result word is written by the
    // solve before it is read
    e = gd::krylov_solve(kc, vals, false, b, x, rtol, max_it);
    if (e != cudaSuccess) return gd::set_error(GD_ERR_CUDA, std::string("krylov launch: ") + cudaGetErrorString(e));
    double out[3];
    e = cudaMemcpyAsync(out, kc.out, sizeof(out), cudaMemcpyDeviceToHost, kc.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(kc.stream);
    if (e != cudaSuccess) return gd::set_error(GD_ERR_CUDA, std::string("result copy: ") + cudaGetErrorString(e));
    if (iterations) *iterations = (int32_t)out[0];
    if (rel_residual) *rel_residual = out[1];
    if (out[2] != 0.0)
        return gd::set_error(GD_ERR_KRYLOV, "gd_solve_noalloc: BiCGStab stopped (status " +
                                                 std::to_string((int)out[2]) + ")");
    return GD_OK;
}
