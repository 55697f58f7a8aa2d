// mess_jk_build_static: the host-buffer J/K build without any device allocation.
//
// mess_jk_build stages D, J and K in device memory it allocates (once per basis, with cudaMalloc) and
// frees when the basis is destroyed.  Some
// callers cannot let the library allocate: a process whose device memory is owned by its own pool
// or arena (an inference server, a framework allocator) and must not see cudaMalloc / cudaFree
// outside it, code on a latency-critical path where cudaFree's implicit device synchronisation is
// not acceptable, or a program that has to keep running when the device is already full.  This
// entry point stages the three matrices in one fixed array that is part of the library image
// instead, so it needs no allocation at call time.
//
// The array holds 3 x 256 x 256 doubles (1.5 MiB) on every GPU that loads the library, until the
// process exits.  Host code cannot use the array's name as a device address (on the host it names a
// host-side stand-in), so the first call on each device looks the address up with
// cudaGetSymbolAddress while that device is current; that first call should therefore come before
// any stream capture.  Every call shares the one array and it keeps the previous call's contents:
// calls that overlap on the GPU (different host threads, or different streams) race on it.
#include <mutex>

#include "mess_internal.h"

#define MESS_STATIC_NMAX 256

static __device__ __align__(256) double g_jk_static[3 * MESS_STATIC_NMAX * MESS_STATIC_NMAX];

namespace {

std::mutex g_static_mu;
double* g_static_ptr[64] = {};   // device address of g_jk_static, per device

mess_status static_workspace(double** out)
{
    int dev = 0;
    MESS_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) { mess_set_error("device index %d out of range", dev); return MESS_EINVAL; }
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_jk_static);
        if (e != cudaSuccess || !p) {
            mess_set_error("cudaGetSymbolAddress of the static J/K workspace failed: %s", cudaGetErrorString(e));
            return MESS_ECUDA;
        }
        g_static_ptr[dev] = static_cast<double*>(p);
    }
    *out = g_static_ptr[dev];
    return MESS_OK;
}

}  // namespace

extern "C" mess_status mess_jk_build_static(const mess_basis* bc, const double* D, double* J, double* K,
                                            const mess_jk_opts* opts, mess_jk_info* info)
{
    mess_basis* b = const_cast<mess_basis*>(bc);
    if (!b || !D || !J || !K) { mess_set_error("null argument"); return MESS_EINVAL; }
    if (b->nmol != 1) { mess_set_error("mess_jk_build_static: single-molecule bases only"); return MESS_EINVAL; }
    const int n = b->nbf;
    if (n > MESS_STATIC_NMAX) {
        mess_set_error("mess_jk_build_static: %d basis functions exceed the static workspace limit of %d",
                       n, MESS_STATIC_NMAX);
        return MESS_EINVAL;
    }
    bool ready = false;
    mess_status st = mess_jk_bins_ready(b, opts, &ready);
    if (st != MESS_OK) return st;
    if (!ready) {
        mess_set_error("mess_jk_build_static: the quartet bins for these options are not built yet; call "
                       "mess_jk_build or mess_jk_build_device once with the same options first");
        return MESS_EINVAL;
    }
    double* w = nullptr;
    st = static_workspace(&w);
    if (st != MESS_OK) return st;
    mess_jk_opts o{};
    if (opts) o = *opts;
    cudaStream_t s = (cudaStream_t)o.cuda_stream;
    const size_t nn = (size_t)n * n;
    double *dD = w, *dJ = w + nn, *dK = w + 2 * nn;
    cudaError_t e = cudaMemcpyAsync(dD, D, nn * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        st = mess_jk_packed(b, dD, dJ, dK, &o, info, /*graphs=*/false);
        if (st == MESS_OK) {
            e = cudaMemcpyAsync(J, dJ, nn * sizeof(double), cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaMemcpyAsync(K, dK, nn * sizeof(double), cudaMemcpyDeviceToHost, s);
        }
    }
    // whatever happened after the first copy was enqueued, the array is free again only once the
    // stream has drained: the next call (on any stream) may then use it
    const cudaError_t es = cudaStreamSynchronize(s);
    if (st != MESS_OK) return st;
    if (e == cudaSuccess) e = es;
    if (e != cudaSuccess) { mess_set_error("mess_jk_build_static: %s", cudaGetErrorString(e)); return MESS_ECUDA; }
    return MESS_OK;
}
