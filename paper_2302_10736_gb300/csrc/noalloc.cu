// noalloc.cu - bus injections by the Ybus method for callers that cannot
// allocate device memory.
//
// Every other entry point of this library works on a pf_grid, whose device
// buffers (including the phasor workspace) are allocated by ybus_build.  Some
// callers cannot call cudaMalloc at all: host frameworks that hand out all
// device memory from their own pool and forbid driver allocations, or
// latency-critical loops in which an allocation (and the device-wide
// synchronization it can imply) is not acceptable.  inj_ybus_noalloc takes a
// Ybus in CSR form that the caller owns (for example the arrays returned by
// ybus_get) and keeps its only scratch, the bus voltage phasors V = vm e^{j va},
// in a file-scope device array of fixed size, so it allocates nothing.
//
// The scratch array is shared by every call in the process on a given device
// and keeps the last call's contents; each call overwrites the entries it
// reads before reading them, so nothing needs clearing.  Calls that overlap on
// the GPU (different streams, no ordering) race on it.
#include <mutex>

#include "pf_internal.h"

namespace pf {

constexpr int kNoAllocMaxBuses = 1 << 18;   // 262,144 buses: 4 MiB of phasor scratch per device

static __device__ __align__(256) double2 g_noalloc_V[kNoAllocMaxBuses];

__global__ void k_noalloc_phasor(int nb, const double *__restrict__ vm, const double *__restrict__ va,
                                 double2 *__restrict__ V)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nb) return;
    double s, c;
    sincos(va[i], &s, &c);
    const double v = vm[i];
    V[i] = make_double2(v * c, v * s);
}

// one thread per Ybus row: I_i = sum_j Y_ij V_j, S_i = V_i conj(I_i) (Eq. 1)
__global__ void k_noalloc_spmv(int nb, const int *__restrict__ rp, const int *__restrict__ ci,
                               const double2 *__restrict__ Y, const double2 *__restrict__ V, double *__restrict__ P,
                               double *__restrict__ Q)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nb) return;
    double Ir = 0.0, Ii = 0.0;
    for (int e = rp[i]; e < rp[i + 1]; ++e) {
        const double2 y = Y[e];
        const double2 v = V[ci[e]];
        Ir = fma(y.x, v.x, Ir);
        Ir = fma(-y.y, v.y, Ir);
        Ii = fma(y.x, v.y, Ii);
        Ii = fma(y.y, v.x, Ii);
    }
    const double2 Vi = V[i];
    P[i] = fma(Vi.x, Ir, Vi.y * Ii);
    Q[i] = fma(Vi.y, Ir, -Vi.x * Ii);
}

// Device address of the scratch array on the current device, looked up once
// per device (with that device current) and cached.
static pf_status noalloc_scratch(double2 **out)
{
    static std::mutex mu;
    static double2 *ptr[256] = {nullptr};
    int dev = 0;
    PF_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 256) return set_error(PF_EUNSUPPORTED, "inj_ybus_noalloc: device ordinal %d", dev);
    std::lock_guard<std::mutex> lk(mu);
    if (!ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_V);
        if (e != cudaSuccess) return cuda_error(e, "inj_ybus_noalloc: cudaGetSymbolAddress");
        ptr[dev] = static_cast<double2 *>(p);
    }
    *out = ptr[dev];
    return PF_OK;
}

}  // namespace pf

using namespace pf;

PF_API pf_status inj_ybus_noalloc(int32_t nb, const int32_t *rowptr, const int32_t *colidx, const double *yval,
                                  const double *vm, const double *va, double *P, double *Q, pf_stream stream)
{
    if (nb < 0) return set_error(PF_EINVAL, "inj_ybus_noalloc: nb = %d", nb);
    if (nb > kNoAllocMaxBuses)
        return set_error(PF_EUNSUPPORTED,
                         "inj_ybus_noalloc: nb = %d exceeds the %d-bus limit of its fixed scratch array", nb,
                         kNoAllocMaxBuses);
    if (nb == 0) return PF_OK;
    if (!rowptr || !colidx || !yval || !vm || !va || !P || !Q)
        return set_error(PF_EINVAL, "inj_ybus_noalloc: NULL pointer");
    if ((uintptr_t)yval & 15u) return set_error(PF_EINVAL, "inj_ybus_noalloc: yval must be 16-byte aligned");
    double2 *V = nullptr;
    pf_status st = noalloc_scratch(&V);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const int blk = 256, grid = (nb + blk - 1) / blk;
    k_noalloc_phasor<<<grid, blk, 0, s>>>(nb, vm, va, V);
    PF_CUDA(cudaGetLastError());
    k_noalloc_spmv<<<grid, blk, 0, s>>>(nb, rowptr, colidx, reinterpret_cast<const double2 *>(yval), V, P, Q);
    PF_CUDA(cudaGetLastError());
    return PF_OK;
}
