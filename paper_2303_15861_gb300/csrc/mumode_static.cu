// adr_mumode_apply_static: the FP64 mu-mode chain y = v x_1 M_1 x_2 M_2 (x_3 M_3) for callers
// that must not call cudaMalloc (for example a host application whose device memory is all
// reserved up front by its own pool, or a pipeline in which an allocation would synchronise
// the device). The intermediates of the chain live in a file-scope device array instead of
// library workspace; the caller provides the factors, the input and the output.
//
// Scratch: two buffers of kStaticScratchElems doubles (2 x 8 MiB), which every GPU that loads
// the library keeps until the process exits. All calls share them, so calls that overlap on
// the GPU (different streams, or different host threads) race; the contents of the last
// call remain. Every intermediate element is written before it is read, so nothing needs
// clearing.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/adr.h"
#include "adr_internal.h"

namespace {

constexpr long long kStaticScratchElems = 1LL << 20;   // per buffer: 1,048,576 doubles
constexpr int kMaxDevices = 64;

__device__ __align__(256) double g_static_scratch[2][kStaticScratchElems];

std::mutex g_static_mutex;
double* g_static_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device. In host code the array's
// name is only a host-side stand-in, so the address is looked up once per device (with that
// device current) and cached.
adr_status static_scratch(double** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return ADR_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return ADR_ERR_ARG;
    std::lock_guard<std::mutex> lock(g_static_mutex);
    if (!g_static_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return ADR_ERR_CUDA;
        g_static_ptr[dev] = static_cast<double*>(p);
    }
    *out = g_static_ptr[dev];
    return ADR_OK;
}

}  // namespace

extern "C" adr_status adr_mumode_apply_static(int dim, const int n[3], const double* const factors[3],
                                              const double* v_dev, double* y_dev, void* cuda_stream) {
    if (dim != 2 && dim != 3) return ADR_ERR_ARG;
    if (!n || !factors || !v_dev || !y_dev) return ADR_ERR_ARG;
    if (static_cast<const void*>(v_dev) == static_cast<const void*>(y_dev)) return ADR_ERR_ARG;
    long long N = 1;
    for (int m = 0; m < dim; ++m) {
        if (n[m] < 1 || n[m] > 4096 || !factors[m]) return ADR_ERR_ARG;
        N *= n[m];
    }
    if (N > kStaticScratchElems) return ADR_ERR_ARG;   // larger than the static scratch
    double* scratch = nullptr;
    adr_status st = static_scratch(&scratch);
    if (st != ADR_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);

    // mode mu as a strided batched GEMM over the state viewed as [P][n_mu][Q]
    const double* in = v_dev;
    for (int mu = 1; mu <= dim; ++mu) {
        double* out = (mu == dim) ? y_dev : scratch + (mu - 1) % 2 * kStaticScratchElems;
        const int nm = n[mu - 1];
        long long Q = 1, P = 1;
        for (int nu = 1; nu < mu; ++nu) Q *= n[nu - 1];
        for (int nu = mu + 1; nu <= dim; ++nu) P *= n[nu - 1];
        adr::ContractArgs<double> a;
        if (mu == 1) {
            a.A = in; a.sam = nm; a.sak = 1; a.sab = 0;
            a.B = factors[0]; a.sbk = 1; a.sbn = nm; a.sbb = 0;     // B[k][j] = M[j][k]
            a.C = out; a.scm = nm; a.scn = 1; a.scb = 0;
            a.M = int(P); a.N = nm; a.K = nm; a.batch = 1;
        } else {
            a.A = factors[mu - 1]; a.sam = nm; a.sak = 1; a.sab = 0;
            a.B = in; a.sbk = Q; a.sbn = 1; a.sbb = (long long)nm * Q;
            a.C = out; a.scm = Q; a.scn = 1; a.scb = (long long)nm * Q;
            a.M = nm; a.N = int(Q); a.K = nm; a.batch = int(P);
        }
        a.n1 = n[0];
        a.n2 = n[1];
        if (adr::launch_contract(a, s) != cudaSuccess) return ADR_ERR_CUDA;
        in = out;
    }
    return ADR_OK;
}
