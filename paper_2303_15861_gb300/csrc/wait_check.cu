// The failure path of the bounded device waits, run on purpose: a kernel waits on an mbarrier
// that nothing arrives on, gives up after a short limit, records the code in the context's
// error word and returns. adr_synchronize then reports ADR_ERR_TIMEOUT and clears the word, and
// the context stays usable. No fault, no trap, no unbounded wait.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/adr.h"
#include "adr_internal.h"
#include "tc_common.cuh"

namespace adr {
namespace {
using namespace tc;

constexpr int kProbeCode = 0x800;

__global__ void wait_probe_kernel(int* err, long long limit_cycles) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(smem_u32(&bar), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const long long t0 = clock64();
        bool done = false;
        while (!(done = mbar_try_wait(smem_u32(&bar), 0u)) && clock64() - t0 < limit_cycles) {
        }
        if (!done) atomicOr(err, kProbeCode);
    }
}

}  // namespace

cudaError_t launch_wait_probe(int* err, double limit_ms, cudaStream_t s) {
    // limit in SM cycles at the part's maximum clock (2070 MHz); at a lower clock it lasts longer
    const long long cycles = static_cast<long long>(limit_ms * 2.07e6);
    wait_probe_kernel<<<1, 32, 0, s>>>(err, cycles);
    return cudaGetLastError();
}

}  // namespace adr
