// k_elementwise.cu - element-wise method (Sec. II-B, IV-C) on the GPU.
//
// Evaluation.  Each branch terminal t (owner bus o, other bus q) evaluates
// its flow from two precomputed constants (see k_setup.cu):
//     S_t = v_o^2 conj(Ys_t) + K_t,   K_t = conj(Yc_t) V_o conj(V_q)      (Eqs. 5-6)
// where V_o conj(V_q) = v_o v_q e^{j(theta_o - theta_q)} carries the sine and
// cosine of the angle difference in registers (formed from the per-bus
// phasors, no per-branch trigonometry).  Its 8 partials (16 per branch):
//     dS_t/dtheta_q = -j K_t            dS_t/dv_q = K_t / v_q = conj(Yc_t) V_o conj(U_q)
//     dS_t/dtheta_o = +j K_t            dS_t/dv_o = 2 v_o conj(Ys_t) + K_t / v_o
//
// Reduction (Eq. 7 and the copy-add of Fig. 2, without atomics).  The
// terminals are laid out by bus window (one CTA) and, inside a window, by
// owner bus sorted on terminal count, so a lane owns one bus and every one of
// its terminals: the segmented sum onto the bus and onto its diagonal
// Jacobian slot runs in registers in a fixed order, and each off-diagonal
// slot (o, q) is written by that lane alone (parallel branches, adjacent in
// the layout, are added in order).  The 32 lanes of a warp own buses with
// equally many terminals, so the evaluation runs with all lanes busy and the
// k-th terminals of a warp are read with coalesced loads.
//     S_o           = v_o^2 conj(sum Ys + y_sh,o) + sum K
//     dS_o/dtheta_o = j sum K
//     dS_o/dv_o     = 2 v_o conj(sum Ys + y_sh,o) + (sum K) / v_o
// A window's Jacobian rows are one contiguous slice of each of the P and Q
// halves of J (canonical layout), so the CTA stages its slice in shared
// memory and writes it back with coalesced stores, together with P and Q.
#include "pf_internal.h"

namespace pf {

__global__ void __launch_bounds__(512) k_jac_ew(int nb, int nnz, int window, const int *__restrict__ rp,
                                                const int4 *__restrict__ slot_meta, const int *__restrict__ slot_kd,
                                                const double2 *__restrict__ slot_ysh,
                                                const int2 *__restrict__ warp_meta,
                                                const double2 *__restrict__ ent_ys,
                                                const double2 *__restrict__ ent_yc,
                                                const int2 *__restrict__ ent_nbr, const double4_32a *__restrict__ U,
                                                double *__restrict__ P, double *__restrict__ Q,
                                                double *__restrict__ J)
{
    extern __shared__ double stg[];
    const int w = blockIdx.x;
    const int b0 = w * window, b1 = min(b0 + window, nb);
    const int r0 = rp[b0];
    const int L = 2 * (rp[b1] - r0);
    double *stP = stg + 2 * L;
    double *stQ = stP + window;
    const int slot = w * window + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const int4 meta = slot_meta[slot];
    if (meta.x >= 0) {
        const int o = meta.x, nt = meta.y, lrow = meta.z, d = meta.w;
        const double4_32a uo = U[o];
        const double v = uo.z, iv = uo.w;
        const double Vr = v * uo.x, Vi = v * uo.y;
        const int2 wm = warp_meta[slot >> 5];
        double sKr = 0.0, sKi = 0.0, sYr = 0.0, sYi = 0.0;
        for (int k = 0; k < nt; ++k) {
            const int e = wm.x + 32 * k + lane;
            const double2 ys = ent_ys[e];
            const double2 yc = ent_yc[e];
            const int2 nq = ent_nbr[e];
            const double4_32a uq = U[nq.x];
            const double Er = fma(Vr, uq.x, Vi * uq.y);     // V_o conj(U_q)
            const double Ei = fma(Vi, uq.x, -Vr * uq.y);
            const double Gr = fma(yc.x, Er, yc.y * Ei);     // conj(Yc) E = dS_t/dv_q
            const double Gi = fma(yc.x, Ei, -yc.y * Er);
            const double Kr = uq.z * Gr, Ki = uq.z * Gi;    // K_t = v_q G
            sKr += Kr;
            sKi += Ki;
            sYr += ys.x;
            sYi += ys.y;
            const int pos = lrow + (nq.y & EW_KMASK);
            if (nq.y & EW_ACCUM) {  // second and later branch of a parallel run
                stg[pos] += Ki;
                stg[pos + d] += Gr;
                stg[L + pos] -= Kr;
                stg[L + pos + d] += Gi;
            } else {
                stg[pos] = Ki;           // J11: Re(-j K)
                stg[pos + d] = Gr;       // J12
                stg[L + pos] = -Kr;      // J21: Im(-j K)
                stg[L + pos + d] = Gi;   // J22
            }
        }
        const double2 ysh = slot_ysh[slot];
        const double Ydr = sYr + ysh.x, Ydi = sYi + ysh.y;
        const double v2 = v * v, tv = v + v;
        const int pos = lrow + slot_kd[slot];
        stg[pos] = -sKi;                          // Re(j sum K)
        stg[pos + d] = fma(tv, Ydr, sKr * iv);
        stg[L + pos] = sKr;                       // Im(j sum K)
        stg[L + pos + d] = fma(-tv, Ydi, sKi * iv);
        stP[o - b0] = fma(v2, Ydr, sKr);
        stQ[o - b0] = fma(-v2, Ydi, sKi);
    }
    __syncthreads();
    double *Jp = J + 2 * (long long)r0;
    double *Jq = J + 2 * (long long)nnz + 2 * (long long)r0;
    for (int x = threadIdx.x; x < L; x += blockDim.x) {
        Jp[x] = stg[x];
        Jq[x] = stg[L + x];
    }
    if (P) {
        for (int x = threadIdx.x; x < b1 - b0; x += blockDim.x) {
            P[b0 + x] = stP[x];
            Q[b0 + x] = stQ[x];
        }
    }
}

__global__ void __launch_bounds__(512) k_inj_ew(int nb, int window, const int4 *__restrict__ slot_meta,
                                                const double2 *__restrict__ slot_ysh,
                                                const int2 *__restrict__ warp_meta,
                                                const double2 *__restrict__ ent_ys,
                                                const double2 *__restrict__ ent_yc,
                                                const int2 *__restrict__ ent_nbr, const double *__restrict__ vm,
                                                const double2 *__restrict__ V, double *__restrict__ P,
                                                double *__restrict__ Q)
{
    extern __shared__ double stg[];
    const int w = blockIdx.x;
    const int b0 = w * window, b1 = min(b0 + window, nb);
    double *stP = stg;
    double *stQ = stg + window;
    const int slot = w * window + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const int4 meta = slot_meta[slot];
    if (meta.x >= 0) {
        const int o = meta.x, nt = meta.y;
        const double2 Vo = V[o];
        const int2 wm = warp_meta[slot >> 5];
        double sKr = 0.0, sKi = 0.0, sYr = 0.0, sYi = 0.0;
        for (int k = 0; k < nt; ++k) {
            const int e = wm.x + 32 * k + lane;
            const double2 ys = ent_ys[e];
            const double2 yc = ent_yc[e];
            const double2 Vq = V[ent_nbr[e].x];
            const double Wr = fma(Vo.x, Vq.x, Vo.y * Vq.y);  // V_o conj(V_q)
            const double Wi = fma(Vo.y, Vq.x, -Vo.x * Vq.y);
            sKr += fma(yc.x, Wr, yc.y * Wi);                // conj(Yc) W
            sKi += fma(yc.x, Wi, -yc.y * Wr);
            sYr += ys.x;
            sYi += ys.y;
        }
        const double2 ysh = slot_ysh[slot];
        const double v = vm[o], v2 = v * v;
        stP[o - b0] = fma(v2, sYr + ysh.x, sKr);
        stQ[o - b0] = fma(-v2, sYi + ysh.y, sKi);
    }
    __syncthreads();
    for (int x = threadIdx.x; x < b1 - b0; x += blockDim.x) {
        P[b0 + x] = stP[x];
        Q[b0 + x] = stQ[x];
    }
}

static size_t jac_smem(const Grid *g) { return (size_t)(2 * g->ew.max_L + 2 * g->ew.window) * sizeof(double); }

cudaError_t launch_jac_ew(const Grid *g, const double4_32a *U, double *P, double *Q, double *J, cudaStream_t s)
{
    const EwDev &L = g->ew;
    if (L.nwin == 0) return cudaSuccess;
    const size_t smem = jac_smem(g);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_jac_ew, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k_jac_ew<<<L.nwin, L.window, smem, s>>>(g->nb, g->nnz, L.window, g->rp, L.slot_meta, L.slot_kd, L.slot_ysh,
                                            L.warp_meta, L.ent_ys, L.ent_yc, L.ent_nbr, U, P, Q, J);
    return cudaGetLastError();
}

cudaError_t launch_inj_ew_vm(const Grid *g, const double *vm, const double2 *V, double *P, double *Q, cudaStream_t s)
{
    const EwDev &L = g->ew;
    if (L.nwin == 0) return cudaSuccess;
    k_inj_ew<<<L.nwin, L.window, 2 * L.window * sizeof(double), s>>>(g->nb, L.window, L.slot_meta, L.slot_ysh,
                                                                     L.warp_meta, L.ent_ys, L.ent_yc, L.ent_nbr,
                                                                     vm, V, P, Q);
    return cudaGetLastError();
}

}  // namespace pf
