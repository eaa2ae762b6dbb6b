// reduced.cu - the reduced Newton Jacobian in CSC order and the mismatch
// vector, gathered from the full evaluation (Eq. 2's blocks on the P rows and
// theta columns of PV and PQ buses and the Q rows and v columns of PQ buses).
//
// The paper computes the full Jacobian on the Ybus pattern and names the
// solver that consumes it (a sparse direct solver taking column-major input);
// this file is that interface step.  Because the canonical layout places every
// entry at a closed-form position, the reduced matrix is a fixed selection and
// permutation of the full one: the host builds, once per set of bus types,
// the canonical position of every reduced entry (jmap) in CSC order, and one
// launch gathers the values.  The full values were written by the evaluation
// kernel just before, so the gather reads them from L2; its DRAM traffic is
// the map and the output.
#include <algorithm>
#include <vector>

#include "pf_internal.h"
#include "ptx.cuh"

namespace pf {

namespace {

struct HostReduced {
    int n = 0, npvpq = 0, npq = 0;
    std::vector<int> colptr, rowidx, jmap, fmap;
    std::vector<int> jinv;                       // [4 nnzY] reduced (CSC) index of each canonical position, or -1
    std::vector<int2> binv;                      // [nb] reduced index of the bus's P and Q equation, or -1
};

// Reduced index of full row/column R (R < nb: theta_R / P_R; R >= nb:
// v_{R-nb} / Q_{R-nb}), -1 if not kept; then the CSC pattern by a counting
// sort on the column.  Canonical rows are visited in ascending order and the
// reduced index grows with R, so every column's rows come out ascending.
pf_status host_reduced(const HostTopo &H, const int *bt, HostReduced &R)
{
    const int nb = H.nb;
    std::vector<int> red(2 * (size_t)nb, -1);
    for (int i = 0; i < nb; ++i) {
        if (bt[i] < 1 || bt[i] > 4)
            return set_error(PF_EINVAL, "bus_type[%d] = %d (1 PQ, 2 PV, 3 ref, 4 isolated)", i, bt[i]);
        if (bt[i] == 1 || bt[i] == 2) red[i] = R.npvpq++;
    }
    for (int i = 0; i < nb; ++i)
        if (bt[i] == 1) red[nb + i] = R.npvpq + R.npq++;
    R.n = R.npvpq + R.npq;
    R.fmap.assign(R.n, 0);
    for (int i = 0; i < nb; ++i) {
        if (red[i] >= 0) R.fmap[red[i]] = i;
        if (red[nb + i] >= 0) R.fmap[red[nb + i]] = i;
    }
    R.colptr.assign(R.n + 1, 0);
    for (int Rw = 0; Rw < 2 * nb; ++Rw) {
        if (red[Rw] < 0) continue;
        for (int p = H.jrp[Rw]; p < H.jrp[Rw + 1]; ++p)
            if (red[H.jci[p]] >= 0) R.colptr[red[H.jci[p]] + 1]++;
    }
    for (int c = 0; c < R.n; ++c) R.colptr[c + 1] += R.colptr[c];
    const int nnz = R.colptr[R.n];
    R.rowidx.assign(nnz, 0);
    R.jmap.assign(nnz, 0);
    std::vector<int> fill(R.colptr.begin(), R.colptr.end() - 1);
    for (int Rw = 0; Rw < 2 * nb; ++Rw) {
        if (red[Rw] < 0) continue;
        for (int p = H.jrp[Rw]; p < H.jrp[Rw + 1]; ++p) {
            const int c = red[H.jci[p]];
            if (c < 0) continue;
            R.rowidx[fill[c]] = red[Rw];
            R.jmap[fill[c]++] = p;
        }
    }
    // inverse maps for the fused element-wise path
    R.jinv.assign(H.jci.size(), -1);
    for (int k = 0; k < nnz; ++k) R.jinv[R.jmap[k]] = k;
    R.binv.resize(nb);
    for (int i = 0; i < nb; ++i) R.binv[i] = make_int2(red[i], red[nb + i]);
    return PF_OK;
}

template <class T>
pf_status upload_vec(DevArena &a, T **dst, const std::vector<T> &src, cudaStream_t s)
{
    PF_CUDA(a.alloc(dst, src.size()));
    if (!src.empty()) PF_CUDA(cudaMemcpyAsync(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice, s));
    return PF_OK;
}

// F[0 .. n) and Jr[0 .. nnz) as one index range, kUnroll entries per thread
// per round: their map entries are loaded together (before the wait for the
// evaluation kernel: programmatic dependent launch), then their values, so a
// round costs two load latencies instead of two per entry.
constexpr int kUnroll = 4;

__global__ void __launch_bounds__(256) k_reduce(int n, int npvpq, int nnz, const int *__restrict__ fmap,
                                                const int *__restrict__ jmap, const double *__restrict__ P,
                                                const double *__restrict__ Q, const double *__restrict__ Ps,
                                                const double *__restrict__ Qs, const double *__restrict__ J,
                                                double *__restrict__ F, double *__restrict__ Jr)
{
    const long long total = (long long)n + nnz;
    const long long stride = (long long)gridDim.x * blockDim.x;
    bool waited = false;
    for (long long base = (long long)blockIdx.x * blockDim.x + threadIdx.x; base < total;
         base += kUnroll * stride) {
        int src[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const long long i = base + u * stride;
            src[u] = i < total ? (i < n ? fmap[i] : jmap[i - n]) : 0;
        }
        if (!waited) {
            pdl_wait();
            waited = true;
        }
        double val[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const long long i = base + u * stride;
            if (i < total) val[u] = i < n ? (i < npvpq ? P[src[u]] - Ps[src[u]] : Q[src[u]] - Qs[src[u]]) : J[src[u]];
        }
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const long long i = base + u * stride;
            if (i < total) {
                if (i < n)
                    F[i] = val[u];
                else
                    Jr[i - n] = val[u];
            }
        }
    }
    if (!waited) pdl_wait();   // every thread waits once (a thread with no entry too)
}

}  // namespace

// The gather after a full evaluation into the grid's scratch: F, and the
// reduced values in the order of `map` (CSC).
cudaError_t launch_reduce(Grid *g, const int *map, const double *Pspec, const double *Qspec, double *F, double *Jr,
                          cudaStream_t s)
{
    const long long total = (long long)g->red_n + g->red_nnz;
    int dev = 0, nsm = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev)) || (e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)))
        return e;
    const int blocks = (int)std::max<long long>(1, std::min<long long>((total + 256 * kUnroll - 1) / (256 * kUnroll),
                                                                       8LL * nsm));
    return launch_k(k_reduce, blocks, 256, 0, s, true, g->red_n, g->red_npvpq, (int)g->red_nnz,
                    (const int *)g->red_fmap, map, (const double *)g->red_P, (const double *)g->red_Q, Pspec, Qspec,
                    (const double *)g->red_J, F, Jr);
}

}  // namespace pf

using namespace pf;

PF_API pf_status grid_set_bus_types(pf_grid *grid, const int32_t *bus_type, pf_stream stream)
{
    if (!grid) return set_error(PF_EINVAL, "grid_set_bus_types: grid is NULL");
    Grid *g = &grid->g;
    if (g->nb > 0 && !bus_type) return set_error(PF_EINVAL, "grid_set_bus_types: bus_type is NULL");
    HostReduced R;
    pf_status st = host_reduced(g->topo, bus_type, R);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    PF_CUDA(cudaStreamSynchronize(s));   // no launch may still read the old map
    for (void *p : {(void *)g->red_colptr, (void *)g->red_rowidx, (void *)g->red_jmap, (void *)g->red_fmap,
                    (void *)g->red_jinv,
                    (void *)g->red_binv, (void *)g->nt_F, (void *)g->nt_J, (void *)g->nt_dx})
        if (p) g->arena.release(p);
    g->red_colptr = g->red_rowidx = g->red_jmap = g->red_fmap = nullptr;
    g->red_jinv = nullptr;
    g->red_binv = nullptr;
    g->nt_F = g->nt_J = g->nt_dx = nullptr;   // sized by n and nnz: re-allocated by the next Newton solve
    g->red_set = 0;
    if ((st = upload_vec(g->arena, &g->red_colptr, R.colptr, s)) ||
        (st = upload_vec(g->arena, &g->red_rowidx, R.rowidx, s)) ||
        (st = upload_vec(g->arena, &g->red_jmap, R.jmap, s)) || (st = upload_vec(g->arena, &g->red_fmap, R.fmap, s)) ||
        (st = upload_vec(g->arena, &g->red_jinv, R.jinv, s)) || (st = upload_vec(g->arena, &g->red_binv, R.binv, s)))
        return st;
    if (!g->red_J) {
        double **const out[3] = {&g->red_P, &g->red_Q, &g->red_J};
        const size_t n[3] = {(size_t)g->nb, (size_t)g->nb, 4 * (size_t)g->nnz};
        PF_CUDA(alloc_all(g->arena, out, n));
    }
    g->red_n = R.n;
    g->red_npvpq = R.npvpq;
    g->red_nnz = R.colptr.back();
    PF_CUDA(cudaStreamSynchronize(s));   // R's vectors are freed on return
    lu_release(g);                       // the LU plan belongs to the previous bus types
    g->red_h_colptr = R.colptr;
    g->red_h_rowidx = R.rowidx;
    g->red_h_fmap = R.fmap;
    g->red_set = 1;
    return PF_OK;
}

PF_API pf_status jac_reduced_info(const pf_grid *grid, int32_t *n, int32_t *n_pvpq, int64_t *nnz)
{
    if (!grid) return set_error(PF_EINVAL, "jac_reduced_info: grid is NULL");
    const Grid *g = &grid->g;
    if (!g->red_set) return set_error(PF_EINVAL, "jac_reduced_info: call grid_set_bus_types first");
    if (n) *n = g->red_n;
    if (n_pvpq) *n_pvpq = g->red_npvpq;
    if (nnz) *nnz = g->red_nnz;
    return PF_OK;
}

PF_API pf_status jac_reduced_pattern(const pf_grid *grid, const int32_t **colptr, const int32_t **rowidx)
{
    if (!grid || !colptr || !rowidx) return set_error(PF_EINVAL, "jac_reduced_pattern: NULL argument");
    const Grid *g = &grid->g;
    if (!g->red_set) return set_error(PF_EINVAL, "jac_reduced_pattern: call grid_set_bus_types first");
    *colptr = g->red_colptr;
    *rowidx = g->red_rowidx;
    return PF_OK;
}

PF_API pf_status jac_reduced(pf_grid *grid, int32_t method, const double *vm, const double *va, const double *Pspec,
                             const double *Qspec, double *F, double *Jr, pf_stream stream)
{
    if (!grid) return set_error(PF_EINVAL, "jac_reduced: grid is NULL");
    Grid *g = &grid->g;
    if (!g->red_set) return set_error(PF_EINVAL, "jac_reduced: call grid_set_bus_types first");
    if (method != 0 && method != 1)
        return set_error(PF_EINVAL, "jac_reduced: method must be 0 (Ybus) or 1 (element-wise)");
    if (g->nb == 0 || g->red_n == 0) return PF_OK;
    if (!vm || !va || !Pspec || !Qspec || !F || (g->red_nnz > 0 && !Jr))
        return set_error(PF_EINVAL, "jac_reduced: NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    if (method == 1) {   // one launch: the element-wise kernel writes the reduced system itself
        TraceScope t(g, PF_K_JAC_EW, s);
        PF_CUDA(launch_jac_ew_reduced(g, vm, va, Pspec, Qspec, F, Jr, s));
        return PF_OK;
    }
    pf_status st = jac_ybus(grid, vm, va, g->red_P, g->red_Q, g->red_J, stream);
    if (st) return st;
    TraceScope t(g, PF_K_REDUCE, s);
    PF_CUDA(launch_reduce(g, g->red_jmap, Pspec, Qspec, F, Jr, s));
    return PF_OK;
}
