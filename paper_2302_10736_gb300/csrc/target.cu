// target.cu - Jacobian values into a caller's sparsity pattern (Alg. 2).
//
// The paper assembles the four blocks of Eq. (2) into a pre-allocated J whose
// pattern contains every block's entries and may hold more (series devices
// such as TCSC couple further buses): index arrays P_xy, found once by
// matching row and column coordinates, say where each block entry goes, and
// every evaluation copies the values there.  Here one map covers all four
// blocks: for each position p of the canonical layout (row-major, the P and
// Q halves), the position in the caller's CSC pattern of the same (row,
// column).  The element-wise kernel stores through the map directly
// (k_ew_red); the Ybus method evaluates into scratch and one launch scatters.
#include <algorithm>
#include <vector>

#include "pf_internal.h"

namespace pf {

namespace {

__global__ void __launch_bounds__(256) k_scatter(long long n, const int *__restrict__ map,
                                                 const double *__restrict__ src, double *__restrict__ dst)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        dst[map[i]] = src[i];
}

// The position in the CSC pattern (colptr, rowidx) of every canonical entry,
// by the row of each entry searched in its column (the first match).
pf_status host_target_map(const HostTopo &H, const int32_t *colptr, const int32_t *rowidx, long long nnz,
                          std::vector<int> &map)
{
    const int n2 = 2 * H.nb;
    if (colptr[0] != 0 || colptr[n2] != nnz)
        return set_error(PF_EINVAL, "jac_set_target_pattern: colptr[0] = %d, colptr[2nb] = %d (nnz %lld)", colptr[0],
                         colptr[n2], nnz);
    for (int c = 0; c < n2; ++c)
        if (colptr[c + 1] < colptr[c])
            return set_error(PF_EINVAL, "jac_set_target_pattern: colptr decreases at column %d", c);
    for (long long k = 0; k < nnz; ++k)
        if (rowidx[k] < 0 || rowidx[k] >= n2)
            return set_error(PF_EINVAL, "jac_set_target_pattern: rowidx[%lld] = %d outside [0, %d)", k, rowidx[k], n2);
    map.assign(H.jci.size(), -1);
    for (int R = 0; R < n2; ++R)
        for (int p = H.jrp[R]; p < H.jrp[R + 1]; ++p) {
            const int C = H.jci[p];
            for (int k = colptr[C]; k < colptr[C + 1]; ++k)
                if (rowidx[k] == R) {
                    map[p] = k;
                    break;
                }
            if (map[p] < 0)
                return set_error(PF_EINVAL, "jac_set_target_pattern: the pattern lacks entry (%d, %d) of Eq. (2)", R, C);
        }
    return PF_OK;
}

}  // namespace

}  // namespace pf

using namespace pf;

PF_API pf_status jac_set_target_pattern(pf_grid *grid, const int32_t *colptr, const int32_t *rowidx, int64_t nnz,
                                        pf_stream stream)
{
    if (!grid) return set_error(PF_EINVAL, "jac_set_target_pattern: grid is NULL");
    Grid *g = &grid->g;
    if (!colptr || (nnz > 0 && !rowidx)) return set_error(PF_EINVAL, "jac_set_target_pattern: NULL argument");
    if (nnz < 0) return set_error(PF_EINVAL, "jac_set_target_pattern: nnz = %lld", (long long)nnz);
    if (nnz >= (1LL << 31)) return set_error(PF_EUNSUPPORTED, "jac_set_target_pattern: nnz >= 2^31");
    std::vector<int> map;
    pf_status st = host_target_map(g->topo, colptr, rowidx, nnz, map);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    PF_CUDA(cudaStreamSynchronize(s));   // no launch may still read the old map
    if (g->tgt_map) g->arena.release(g->tgt_map);
    g->tgt_map = nullptr;
    g->tgt_set = 0;
    PF_CUDA(g->arena.alloc(&g->tgt_map, std::max<size_t>(map.size(), 1)));
    if (!map.empty())
        PF_CUDA(cudaMemcpyAsync(g->tgt_map, map.data(), map.size() * sizeof(int), cudaMemcpyHostToDevice, s));
    PF_CUDA(cudaStreamSynchronize(s));   // map is freed on return
    g->tgt_nnz = nnz;
    g->tgt_set = 1;
    return PF_OK;
}

PF_API pf_status jac_target(pf_grid *grid, int32_t method, const double *vm, const double *va, double *P, double *Q,
                            double *Jt, pf_stream stream)
{
    if (!grid) return set_error(PF_EINVAL, "jac_target: grid is NULL");
    Grid *g = &grid->g;
    if (!g->tgt_set) return set_error(PF_EINVAL, "jac_target: call jac_set_target_pattern first");
    if (method != 0 && method != 1) return set_error(PF_EINVAL, "jac_target: method must be 0 (Ybus) or 1 (element-wise)");
    if (g->nb == 0) return PF_OK;
    if (!vm || !va || !Jt) return set_error(PF_EINVAL, "jac_target: NULL argument");
    if ((P == nullptr) != (Q == nullptr)) return set_error(PF_EINVAL, "jac_target: P and Q must both be set or both NULL");
    cudaStream_t s = (cudaStream_t)stream;
    if (method == 1) {   // one launch: the element-wise kernel stores through the map
        TraceScope t(g, PF_K_JAC_EW, s);
        PF_CUDA(launch_jac_ew_mapped(g, vm, va, P, Q, g->tgt_map, Jt, s));
        return PF_OK;
    }
    const long long n = 4LL * g->nnz;
    if (!g->tgt_J) PF_CUDA(g->arena.alloc(&g->tgt_J, (size_t)n));
    pf_status st = jac_ybus(grid, vm, va, P, Q, g->tgt_J, stream);
    if (st) return st;
    int dev = 0, nsm = 0;
    PF_CUDA(cudaGetDevice(&dev));
    PF_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, 8LL * nsm));
    k_scatter<<<blocks, 256, 0, s>>>(n, g->tgt_map, g->tgt_J, Jt);
    PF_CUDA(cudaGetLastError());
    return PF_OK;
}
