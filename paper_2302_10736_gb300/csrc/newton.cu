// newton.cu - Newton-Raphson power flow around the evaluation kernels.
//
// The paper computes the injections and the Jacobian that a Newton step
// needs and hands the Jacobian to a sparse direct solver; this file closes the
// loop on the GPU.  Iteration k: the mismatch F and the reduced Jacobian J_r
// in CSC order (jac_reduced: one launch by the element-wise method), max |F|
// to the host (the only host round trip), then J_r dx = F by the library's
// sparse LU (lu.cu, one cooperative launch) and x <- x - dx, with x the
// angles of the PV and PQ buses and the magnitudes of the PQ buses.
#include <algorithm>
#include <cstring>

#include "pf_internal.h"

namespace pf {

namespace {

// max |F| as the bit pattern of a non-negative double (ordered like the value;
// NaN compares above every finite value, so it never passes a tolerance)
__global__ void __launch_bounds__(256) k_absmax(int n, const double *__restrict__ F, unsigned long long *out)
{
    unsigned long long m = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        m = max(m, (unsigned long long)__double_as_longlong(fabs(F[i])));
    for (int off = 16; off > 0; off >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, off));
    if ((threadIdx.x & 31) == 0 && m) atomicMax(out, m);
}

// x <- x - dx: unknown k < npvpq is the angle of bus fmap[k], the rest the
// magnitude of bus fmap[k]
__global__ void __launch_bounds__(256) k_newton_update(int n, int npvpq, const int *__restrict__ fmap,
                                                       const double *__restrict__ dx, double *vm, double *va)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const int b = fmap[k];
        if (k < npvpq)
            va[b] -= dx[k];
        else
            vm[b] -= dx[k];
    }
}

}  // namespace

}  // namespace pf

using namespace pf;

PF_API pf_status powerflow_newton(pf_grid *grid, int32_t method, double *vm, double *va, const double *Pspec,
                                  const double *Qspec, double tol, int32_t max_iter, int32_t *iterations,
                                  double *mismatch, pf_stream stream)
{
    if (!grid) return set_error(PF_EINVAL, "powerflow_newton: grid is NULL");
    Grid *g = &grid->g;
    if (!g->red_set) return set_error(PF_EINVAL, "powerflow_newton: call grid_set_bus_types first");
    if (method != 0 && method != 1)
        return set_error(PF_EINVAL, "powerflow_newton: method must be 0 (Ybus) or 1 (element-wise)");
    if (!(tol >= 0.0) || max_iter < 0) return set_error(PF_EINVAL, "powerflow_newton: tol < 0 or max_iter < 0");
    if (iterations) *iterations = 0;
    if (mismatch) *mismatch = 0.0;
    const int n = g->red_n;
    const long long nnz = g->red_nnz;
    if (g->nb == 0 || n == 0) return PF_OK;
    if (!vm || !va || !Pspec || !Qspec) return set_error(PF_EINVAL, "powerflow_newton: NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    if (!g->nt_dx) {
        double **const out[3] = {&g->nt_F, &g->nt_J, &g->nt_dx};
        const size_t sz[3] = {(size_t)n, (size_t)std::max<long long>(nnz, 1), (size_t)n};
        PF_CUDA(alloc_all(g->arena, out, sz));
    }
    if (!g->nt_max) PF_CUDA(g->arena.alloc(&g->nt_max, 1));
    if (pf_status st = lu_prepare(g, s)) return st;
    int dev = 0, nsm = 0;
    PF_CUDA(cudaGetDevice(&dev));
    PF_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = std::max(1, std::min((n + 255) / 256, 4 * nsm));
    for (int it = 0;; ++it) {
        pf_status st = jac_reduced(grid, method, vm, va, Pspec, Qspec, g->nt_F, g->nt_J, stream);
        if (st) return st;
        PF_CUDA(cudaMemsetAsync(g->nt_max, 0, sizeof(unsigned long long), s));
        k_absmax<<<blocks, 256, 0, s>>>(n, g->nt_F, g->nt_max);
        PF_CUDA(cudaGetLastError());
        unsigned long long bits = 0;
        int derr = 0;
        PF_CUDA(cudaMemcpyAsync(&bits, g->nt_max, sizeof(bits), cudaMemcpyDeviceToHost, s));
        PF_CUDA(cudaMemcpyAsync(&derr, g->err, sizeof(int), cudaMemcpyDeviceToHost, s));
        PF_CUDA(cudaStreamSynchronize(s));
        if (derr == DEV_SINGULAR) {   // the previous iteration's factorization met a zero pivot
            PF_CUDA(cudaMemsetAsync(g->err, 0, sizeof(int), s));
            PF_CUDA(cudaStreamSynchronize(s));
            return set_error(PF_ENOCONV, "powerflow_newton: zero or non-finite pivot in the reduced Jacobian's LU "
                                         "at iteration %d", it - 1);
        }
        if (derr != DEV_OK) return grid_check_error(grid, stream);
        double fmax;
        std::memcpy(&fmax, &bits, sizeof(fmax));
        if (iterations) *iterations = it;
        if (mismatch) *mismatch = fmax;
        if (fmax <= tol) return PF_OK;
        if (it == max_iter)
            return set_error(PF_ENOCONV, "powerflow_newton: max |F| = %g after %d iterations (tol %g)", fmax, it,
                             tol);
        {
            TraceScope t(g, PF_K_LU, s);
            PF_CUDA(launch_lu_solve(g, g->nt_J, g->nt_F, g->nt_dx, s));
        }
        k_newton_update<<<blocks, 256, 0, s>>>(n, g->red_npvpq, g->red_fmap, g->nt_dx, vm, va);
        PF_CUDA(cudaGetLastError());
    }
}
