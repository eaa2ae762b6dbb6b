// k_study.cu - the paper's two-step structure of the element-wise method on
// the GPU, for comparison with the fused kernel of k_elementwise.cu.
//
// The paper evaluates every line's flows and 16 partials in one vectorised
// pass into an intermediate array (Sec. IV-C.1), then assembles them onto the
// buses and the Jacobian slots in a separate pass (Sec. IV-C.2, Figs. 2-3),
// and names that assembly the bottleneck.  Here the same split runs as three
// launches: the phasor step (k_phasor), the evaluation of every sorted
// terminal into K_t and G_t (the 8 partials of a terminal follow from them:
// -jK, G off the diagonal, jK and K / v_o onto it), and one of two assembly
// strategies:
//   gather     one thread per bus walks its terminals in sorted order: its
//              Jacobian row's off-diagonal slots (parallel runs added in
//              order), then the diagonal and S - deterministic, no atomics;
//   copy-add   the per-bus constants first (2 v conj(Yd), v^2 conj(Yd) and
//              zeros elsewhere), then one thread per terminal adds its
//              contributions with floating-point atomics - the order of the
//              additions varies from run to run.
// Only the study entry point jac_elementwise_study uses these kernels.
//
// The paper also compares storing complex voltages interleaved (re, im pairs)
// against separate real and imaginary arrays for its Ybus power calculation
// (Sec. IV-B.1, Table I).  inj_ybus_study runs the phasor step and a
// one-row-per-thread CSR SpMV with either layout, the arithmetic otherwise
// identical.
#include "fastmath.cuh"
#include "pf_internal.h"
#include "ptx.cuh"

namespace pf {

namespace {

__global__ void __launch_bounds__(256) k_ts_eval(int T, const double2 *__restrict__ tcoup,
                                                 const int2 *__restrict__ tnbr, const int *__restrict__ town,
                                                 const double4_32a *__restrict__ U, const double2 *__restrict__ V,
                                                 double4_32a *__restrict__ KG)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= T) return;
    const double2 yc = tcoup[p];
    const double2 Vo = V[town[p]];
    const double4_32a uq = U[tnbr[p].x];
    const double Er = fma(Vo.x, uq.x, Vo.y * uq.y);   // V_o conj(U_q)
    const double Ei = fma(Vo.y, uq.x, -Vo.x * uq.y);
    const double Gr = fma(yc.x, Er, yc.y * Ei);       // conj(Yc) E = dS_t/dv_q
    const double Gi = fma(yc.x, Ei, -yc.y * Er);
    KG[p] = make_double4_32a(uq.z * Gr, uq.z * Gi, Gr, Gi);   // K_t = v_q G, G
}

// one thread per bus: its terminals in sorted order
__global__ void __launch_bounds__(256) k_ts_gather(int nb, int nnz, const int *__restrict__ rp,
                                                   const int *__restrict__ kd, const int *__restrict__ tp,
                                                   const int2 *__restrict__ tnbr, const double2 *__restrict__ yd,
                                                   const double4_32a *__restrict__ U,
                                                   const double4_32a *__restrict__ KG, double *__restrict__ P,
                                                   double *__restrict__ Q, double *__restrict__ J)
{
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= nb) return;
    const int rs = rp[o], d = rp[o + 1] - rs, base = 2 * rs;
    double *J1 = J + base, *J2 = J + 2LL * nnz + base;
    double sKr = 0.0, sKi = 0.0;
    for (int p = tp[o]; p < tp[o + 1]; ++p) {
        const double4_32a kg = KG[p];
        sKr += kg.x;
        sKi += kg.y;
        const int y = tnbr[p].y, pos = y & EW_KMASK;
        if (y & EW_ACCUM) {   // later branch of a parallel run
            J1[pos] += kg.y;
            J1[pos + d] += kg.z;
            J2[pos] -= kg.x;
            J2[pos + d] += kg.w;
        } else {
            J1[pos] = kg.y;        // Re(-j K)
            J1[pos + d] = kg.z;    // Re G
            J2[pos] = -kg.x;       // Im(-j K)
            J2[pos + d] = kg.w;    // Im G
        }
    }
    const double4_32a uo = U[o];
    const double2 y = yd[o];
    const double v = uo.z, iv = uo.w, v2 = v * v, tv = v + v;
    const int pos = kd[o];
    J1[pos] = -sKi;
    J1[pos + d] = fma(tv, y.x, sKr * iv);
    J2[pos] = sKr;
    J2[pos + d] = fma(-tv, y.y, sKi * iv);
    if (P) {
        P[o] = fma(v2, y.x, sKr);
        Q[o] = fma(-v2, y.y, sKi);
    }
}

// copy-add, step 1: the bus constants (the rest of the slots were zeroed)
__global__ void __launch_bounds__(256) k_ts_init(int nb, int nnz, const int *__restrict__ rp,
                                                 const int *__restrict__ kd, const double2 *__restrict__ yd,
                                                 const double4_32a *__restrict__ U, double *__restrict__ P,
                                                 double *__restrict__ Q, double *__restrict__ J)
{
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= nb) return;
    const int rs = rp[o], d = rp[o + 1] - rs, pos = 2 * rs + kd[o];
    const double2 y = yd[o];
    const double v = U[o].z, v2 = v * v, tv = v + v;
    J[pos + d] = tv * y.x;
    J[2LL * nnz + pos + d] = -tv * y.y;
    P[o] = v2 * y.x;
    Q[o] = -v2 * y.y;
}

// copy-add, step 2: every terminal adds onto its off-diagonal slot and onto
// its owner's diagonal slots and injection
__global__ void __launch_bounds__(256) k_ts_atomic(int T, int nnz, const int *__restrict__ rp,
                                                   const int *__restrict__ kd, const int2 *__restrict__ tnbr,
                                                   const int *__restrict__ town, const double4_32a *__restrict__ U,
                                                   const double4_32a *__restrict__ KG, double *__restrict__ P,
                                                   double *__restrict__ Q, double *__restrict__ J)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= T) return;
    const double4_32a kg = KG[p];
    const int o = town[p], rs = rp[o], d = rp[o + 1] - rs, base = 2 * rs;
    double *J1 = J + base, *J2 = J + 2LL * nnz + base;
    const int pos = tnbr[p].y & EW_KMASK, pd = kd[o];
    const double iv = U[o].w;
    atomicAdd(&J1[pos], kg.y);
    atomicAdd(&J1[pos + d], kg.z);
    atomicAdd(&J2[pos], -kg.x);
    atomicAdd(&J2[pos + d], kg.w);
    atomicAdd(&J1[pd], -kg.y);
    atomicAdd(&J1[pd + d], kg.x * iv);
    atomicAdd(&J2[pd], kg.x);
    atomicAdd(&J2[pd + d], kg.y * iv);
    atomicAdd(&P[o], kg.x);
    atomicAdd(&Q[o], kg.y);
}

// V = v e^{j theta} as interleaved pairs (SEP = false) or separate arrays
template <bool SEP>
__global__ void __launch_bounds__(256) k_vs_phasor(int nb, const double *__restrict__ vm,
                                                   const double *__restrict__ va, const ITrig *__restrict__ trig,
                                                   double *__restrict__ V)
{
    __shared__ ITrig tab[kITrigN];
    for (int k = threadIdx.x; k < kITrigN; k += blockDim.x)
        tab[k] = trig[(blockIdx.x % kITrigCopies) * kITrigN + k];
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nb) return;
    double s, c;
    int_sincos(va[i], tab, &s, &c);
    const double v = vm[i];
    if (SEP) {
        V[i] = v * c;
        V[nb + i] = v * s;
    } else {
        reinterpret_cast<double2 *>(V)[i] = make_double2(v * c, v * s);
    }
}

// S_i = V_i conj(sum_j Y_ij V_j), one row per thread
template <bool SEP>
__global__ void __launch_bounds__(256) k_vs_spmv(int nb, const int *__restrict__ rp, const int *__restrict__ ci,
                                                 const double2 *__restrict__ Y, const double *__restrict__ V,
                                                 double *__restrict__ P, double *__restrict__ Q)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nb) return;
    const double2 *V2 = reinterpret_cast<const double2 *>(V);
    double Ir = 0.0, Ii = 0.0;
    for (int e = rp[i]; e < rp[i + 1]; ++e) {
        const int j = ci[e];
        const double2 y = Y[e];
        const double vr = SEP ? V[j] : V2[j].x, vi = SEP ? V[nb + j] : V2[j].y;
        Ir = fma(y.x, vr, Ir);
        Ir = fma(-y.y, vi, Ir);
        Ii = fma(y.x, vi, Ii);
        Ii = fma(y.y, vr, Ii);
    }
    const double vr = SEP ? V[i] : V2[i].x, vi = SEP ? V[nb + i] : V2[i].y;
    P[i] = fma(vr, Ir, vi * Ii);
    Q[i] = fma(vi, Ir, -vr * Ii);
}

}  // namespace

}  // namespace pf

using namespace pf;

PF_API pf_status inj_ybus_study(pf_grid *grid, int32_t separate, const double *vm, const double *va, double *P,
                                double *Q, pf_stream stream)
{
    if (!grid) return set_error(PF_EINVAL, "inj_ybus_study: grid is NULL");
    Grid *g = &grid->g;
    if (separate != 0 && separate != 1) return set_error(PF_EINVAL, "inj_ybus_study: separate must be 0 or 1");
    if (g->nb == 0) return PF_OK;
    if (!vm || !va || !P || !Q) return set_error(PF_EINVAL, "inj_ybus_study: NULL argument");
    const int nb = g->nb;
    cudaStream_t s = (cudaStream_t)stream;
    if (!g->vs_V) PF_CUDA(g->arena.alloc(&g->vs_V, 2 * (size_t)nb));
    const int blocks = (nb + 255) / 256;
    if (separate) {
        k_vs_phasor<true><<<blocks, 256, 0, s>>>(nb, vm, va, trig_table(), g->vs_V);
        k_vs_spmv<true><<<blocks, 256, 0, s>>>(nb, g->rp, g->ci, g->yv, g->vs_V, P, Q);
    } else {
        k_vs_phasor<false><<<blocks, 256, 0, s>>>(nb, vm, va, trig_table(), g->vs_V);
        k_vs_spmv<false><<<blocks, 256, 0, s>>>(nb, g->rp, g->ci, g->yv, g->vs_V, P, Q);
    }
    PF_CUDA(cudaGetLastError());
    return PF_OK;
}

PF_API pf_status jac_elementwise_study(pf_grid *grid, int32_t strategy, const double *vm, const double *va,
                                       double *P, double *Q, double *J, pf_stream stream)
{
    if (!grid) return set_error(PF_EINVAL, "jac_elementwise_study: grid is NULL");
    Grid *g = &grid->g;
    if (strategy != 0 && strategy != 1)
        return set_error(PF_EINVAL, "jac_elementwise_study: strategy must be 0 (gather) or 1 (copy-add)");
    if (g->nb == 0) return PF_OK;
    if (!vm || !va || !J || !P || !Q) return set_error(PF_EINVAL, "jac_elementwise_study: NULL argument");
    const int T = 2 * g->nl, nb = g->nb;
    cudaStream_t s = (cudaStream_t)stream;
    if (!g->ts_KG && T > 0) PF_CUDA(g->arena.alloc(&g->ts_KG, (size_t)T));
    PF_CUDA(launch_phasor(nb, vm, va, g->ph_u, g->ph_v, s));
    if (T > 0) {
        k_ts_eval<<<(T + 255) / 256, 256, 0, s>>>(T, g->tcoup, g->tnbr, g->town, g->ph_u, g->ph_v, g->ts_KG);
        PF_CUDA(cudaGetLastError());
    }
    if (strategy == 0) {
        k_ts_gather<<<(nb + 255) / 256, 256, 0, s>>>(nb, g->nnz, g->rp, g->kd, g->tp, g->tnbr, g->bus_yd, g->ph_u,
                                                      g->ts_KG, P, Q, J);
        PF_CUDA(cudaGetLastError());
        return PF_OK;
    }
    PF_CUDA(cudaMemsetAsync(J, 0, 4 * (size_t)g->nnz * sizeof(double), s));
    k_ts_init<<<(nb + 255) / 256, 256, 0, s>>>(nb, g->nnz, g->rp, g->kd, g->bus_yd, g->ph_u, P, Q, J);
    PF_CUDA(cudaGetLastError());
    if (T > 0) {
        k_ts_atomic<<<(T + 255) / 256, 256, 0, s>>>(T, g->nnz, g->rp, g->kd, g->tnbr, g->town, g->ph_u, g->ts_KG, P,
                                                     Q, J);
        PF_CUDA(cudaGetLastError());
    }
    return PF_OK;
}
