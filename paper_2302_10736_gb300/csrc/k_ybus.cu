// k_ybus.cu - Ybus method on the CSR admittance matrix (Sec. II-A, IV-B).
//
// W lanes serve one Ybus row (W = 1 .. 32, the "vector CSR" family; W = 32 is
// the warp-per-row SpMV).  Rows are independent, so the two passes of Alg. 1
// (pass 1: I = Ybus V and the products Y_ij V_j, Y_ij U_j; pass 2: the
// diag(V) and diag(I) corrections) fuse into one sweep per row: only the
// diagonal entry needs the finished row current I_i, and it is completed by
// the lane that holds it after a W-lane shuffle reduction.
//
// Per structural (i, j), with U_j = e^{j theta_j} and YU = Y_ij U_j:
//     dS_i/dv_j     = V_i conj(YU)                               (Eq. 4)
//     dS_i/dtheta_j = -j V_i conj(Y_ij V_j) = -j v_j dS_i/dv_j    (Eq. 3)
//     I_i          += v_j YU
// and on the diagonal additionally  +j V_i conj(I_i)  and  +conj(I_i) U_i.
// (Alg. 1 as printed carries the opposite sign on dS/dtheta; Eq. 3 is used.)
// Values are written straight into the canonical J layout, i.e. the copy of
// Alg. 2 with its index arrays in closed form.
//
// The row's first column indices (topology) are loaded before the
// programmatic-dependent-launch wait; the phasor gathers of a chunk are issued
// together before its arithmetic.
//
// Two forms: the paper's step 1 as its own launch (k_phasor writes U, V for
// every bus, the row kernels gather them), or fused (k_ybus_fused: each lane
// forms the phasors of its entries' columns from vm, va itself, with the
// integer-pipe sine/cosine of isincos.cuh, so one launch evaluates and nothing
// goes through memory in between; a bus's phasor is formed once per entry of
// its column, about 3.5 times on these grids).
#include "fastmath.cuh"
#include "pf_internal.h"
#include "ptx.cuh"

namespace pf {

// entries per lane prefetched together: a row of the synthetic grids has about 3.5
// entries, so wide rows (W >= 4 lanes) hold one each and narrow ones several
template <int W>
constexpr int kChunkW = W >= 4 ? 1 : (W == 2 ? 2 : 4);

template <int W>
__global__ void __launch_bounds__(512) k_inj_ybus(int nb, const int *__restrict__ yrow, const int *__restrict__ rp,
                                                   const int *__restrict__ ci,
                                                   const double2 *__restrict__ Y, const double2 *__restrict__ V,
                                                   double *__restrict__ P, double *__restrict__ Q)
{
    pdl_launch_dependents();   // the next evaluation's phasor launch may start (it waits for this grid)
    const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int grp = (int)(gid / W), lane = (int)(gid % W);
    const bool valid = grp < nb;
    const int row = valid ? yrow[grp] : 0;
    int rs = 0, d = 0;
    int jj[kChunkW<W>];
    double2 yy[kChunkW<W>];
    if (valid) {
        rs = rp[row];
        d = rp[row + 1] - rs;
    }
#pragma unroll
    for (int j = 0; j < kChunkW<W>; ++j) {
        const int k = lane + W * j;
        if (k < d) jj[j] = ci[rs + k];
    }
    pdl_wait();
#pragma unroll
    for (int j = 0; j < kChunkW<W>; ++j) {
        const int k = lane + W * j;
        if (k < d) yy[j] = Y[rs + k];   // parameter-dependent: after the wait
    }
    double Ir = 0.0, Ii = 0.0;
    for (int k0 = lane; k0 < d; k0 += W * kChunkW<W>) {
        if (k0 != lane) {
#pragma unroll
            for (int j = 0; j < kChunkW<W>; ++j) {
                const int k = k0 + W * j;
                if (k < d) {
                    jj[j] = ci[rs + k];
                    yy[j] = Y[rs + k];
                }
            }
        }
        double2 vv[kChunkW<W>];
#pragma unroll
        for (int j = 0; j < kChunkW<W>; ++j)
            if (k0 + W * j < d) vv[j] = V[jj[j]];
#pragma unroll
        for (int j = 0; j < kChunkW<W>; ++j) {
            if (k0 + W * j < d) {
                Ir = fma(yy[j].x, vv[j].x, Ir);
                Ir = fma(-yy[j].y, vv[j].y, Ir);
                Ii = fma(yy[j].x, vv[j].y, Ii);
                Ii = fma(yy[j].y, vv[j].x, Ii);
            }
        }
    }
#pragma unroll
    for (int off = W / 2; off > 0; off >>= 1) {
        Ir += __shfl_xor_sync(0xffffffffu, Ir, off, W);
        Ii += __shfl_xor_sync(0xffffffffu, Ii, off, W);
    }
    if (valid && lane == 0) {
        const double2 Vi = V[row];
        P[row] = fma(Vi.x, Ir, Vi.y * Ii);   // S = V conj(I)
        Q[row] = fma(Vi.y, Ir, -Vi.x * Ii);
    }
}

template <int W>
__global__ void __launch_bounds__(512) k_jac_ybus(int nb, int nnz, const int *__restrict__ yrow,
                                                   const int *__restrict__ rp,
                                                   const int *__restrict__ ci, const double2 *__restrict__ Y,
                                                   const double4_32a *__restrict__ U, double *__restrict__ P,
                                                   double *__restrict__ Q, double *__restrict__ J)
{
    pdl_launch_dependents();   // the next evaluation's phasor launch may start (it waits for this grid)
    const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int grp = (int)(gid / W), lane = (int)(gid % W);
    const bool valid = grp < nb;
    const int row = valid ? yrow[grp] : 0;
    int rs = 0, d = 0;
    int jj[kChunkW<W>];
    double2 yy[kChunkW<W>];
    if (valid) {
        rs = rp[row];
        d = rp[row + 1] - rs;
    }
#pragma unroll
    for (int j = 0; j < kChunkW<W>; ++j) {
        const int k = lane + W * j;
        if (k < d) jj[j] = ci[rs + k];
    }
    pdl_wait();
#pragma unroll
    for (int j = 0; j < kChunkW<W>; ++j) {
        const int k = lane + W * j;
        if (k < d) yy[j] = Y[rs + k];   // parameter-dependent: after the wait
    }
    double Ir = 0.0, Ii = 0.0;
    double dTr = 0.0, dTi = 0.0, dVr = 0.0, dVi = 0.0;  // diagonal partials (lane that owns it)
    int kd = -1;
    double4_32a ui = make_double4_32a(0.0, 0.0, 0.0, 0.0);
    if (valid) ui = U[row];
    const double Vr = ui.z * ui.x, Vi = ui.z * ui.y;
    for (int k0 = lane; k0 < d; k0 += W * kChunkW<W>) {
        if (k0 != lane) {
#pragma unroll
            for (int j = 0; j < kChunkW<W>; ++j) {
                const int k = k0 + W * j;
                if (k < d) {
                    jj[j] = ci[rs + k];
                    yy[j] = Y[rs + k];
                }
            }
        }
        double4_32a uu[kChunkW<W>];
#pragma unroll
        for (int j = 0; j < kChunkW<W>; ++j)
            if (k0 + W * j < d) uu[j] = U[jj[j]];
#pragma unroll
        for (int j = 0; j < kChunkW<W>; ++j) {
            const int k = k0 + W * j;
            if (k < d) {
                const double YUr = fma(yy[j].x, uu[j].x, -yy[j].y * uu[j].y);
                const double YUi = fma(yy[j].x, uu[j].y, yy[j].y * uu[j].x);
                const double sVr = fma(Vr, YUr, Vi * YUi);    // V_i conj(YU)
                const double sVi = fma(Vi, YUr, -Vr * YUi);
                const double vj = uu[j].z;
                Ir = fma(vj, YUr, Ir);
                Ii = fma(vj, YUi, Ii);
                const double sTr = vj * sVi, sTi = -vj * sVr;   // -j v_j dS/dv_j
                if (jj[j] == row) {
                    kd = k;
                    dTr = sTr;
                    dTi = sTi;
                    dVr = sVr;
                    dVi = sVi;
                } else {
                    const int p = 2 * rs + k;
                    J[p] = sTr;
                    J[p + d] = sVr;
                    J[2 * nnz + p] = sTi;
                    J[2 * nnz + p + d] = sVi;
                }
            }
        }
    }
#pragma unroll
    for (int off = W / 2; off > 0; off >>= 1) {
        Ir += __shfl_xor_sync(0xffffffffu, Ir, off, W);
        Ii += __shfl_xor_sync(0xffffffffu, Ii, off, W);
    }
    if (!valid) return;
    const double Sr = fma(Vr, Ir, Vi * Ii), Si = fma(Vi, Ir, -Vr * Ii);
    if (kd >= 0) {
        dTr -= Si;                           // + j S_i  (= j V_i conj(I_i))
        dTi += Sr;
        dVr += fma(Ir, ui.x, Ii * ui.y);     // + conj(I_i) U_i
        dVi += fma(Ir, ui.y, -Ii * ui.x);
        const int p = 2 * rs + kd;
        J[p] = dTr;
        J[p + d] = dVr;
        J[2 * nnz + p] = dTi;
        J[2 * nnz + p + d] = dVi;
    }
    if (lane == 0 && P) {
        P[row] = Sr;
        Q[row] = Si;
    }
}

// Injections (JAC = false) or injections and Jacobian (JAC = true) with the
// phasor step fused: W lanes per row, each forming U_j = e^{j theta_j}, v_j for
// its entries and the row's own V_i.
template <int W, bool JAC>
__global__ void __launch_bounds__(512) k_ybus_fused(int nb, int nnz, const int *__restrict__ yrow,
                                                     const int *__restrict__ rp,
                                                     const int *__restrict__ ci, const double2 *__restrict__ Y,
                                                     const double *__restrict__ vm, const double *__restrict__ va,
                                                     const ITrig *__restrict__ trig, double *__restrict__ P,
                                                     double *__restrict__ Q, double *__restrict__ J)
{
    __shared__ ITrig tab[kITrigN];
    pdl_launch_dependents();
    const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int grp = (int)(gid / W), lane = (int)(gid % W);
    const bool valid = grp < nb;
    const int row = valid ? yrow[grp] : 0;
    int rs = 0, d = 0;
    int jj[kChunkW<W>];
    if (valid) {
        rs = rp[row];
        d = rp[row + 1] - rs;
    }
#pragma unroll
    for (int j = 0; j < kChunkW<W>; ++j) {
        const int k = lane + W * j;
        if (k < d) jj[j] = ci[rs + k];
    }
    for (int k = threadIdx.x; k < kITrigN; k += blockDim.x) tab[k] = trig[(blockIdx.x % kITrigCopies) * kITrigN + k];
    pdl_wait();   // the state and the Ybus values may be the previous kernel's
    double2 yy[kChunkW<W>];
#pragma unroll
    for (int j = 0; j < kChunkW<W>; ++j) {
        const int k = lane + W * j;
        if (k < d) yy[j] = Y[rs + k];
    }
    const double thi = valid ? va[row] : 0.0, vi = valid ? vm[row] : 0.0;
    __syncthreads();   // the table
    double si, cs;
    int_sincos(thi, tab, &si, &cs);
    const double Vr = vi * cs, Vi = vi * si;
    double Ir = 0.0, Ii = 0.0;
    double dTr = 0.0, dTi = 0.0, dVr = 0.0, dVi = 0.0;   // diagonal partials (lane that owns it)
    int kd = -1;
    for (int k0 = lane; k0 < d; k0 += W * kChunkW<W>) {
        if (k0 != lane) {
#pragma unroll
            for (int j = 0; j < kChunkW<W>; ++j) {
                const int k = k0 + W * j;
                if (k < d) {
                    jj[j] = ci[rs + k];
                    yy[j] = Y[rs + k];
                }
            }
        }
        double thj[kChunkW<W>], vj[kChunkW<W>];
#pragma unroll
        for (int j = 0; j < kChunkW<W>; ++j)
            if (k0 + W * j < d) {
                thj[j] = va[jj[j]];
                vj[j] = vm[jj[j]];
            }
#pragma unroll
        for (int j = 0; j < kChunkW<W>; ++j) {
            const int k = k0 + W * j;
            if (k < d) {
                double s, c;
                int_sincos(thj[j], tab, &s, &c);
                if (JAC) {
                    const double YUr = fma(yy[j].x, c, -yy[j].y * s);   // Y_ij U_j
                    const double YUi = fma(yy[j].x, s, yy[j].y * c);
                    const double sVr = fma(Vr, YUr, Vi * YUi);          // V_i conj(YU)
                    const double sVi = fma(Vi, YUr, -Vr * YUi);
                    Ir = fma(vj[j], YUr, Ir);
                    Ii = fma(vj[j], YUi, Ii);
                    const double sTr = vj[j] * sVi, sTi = -vj[j] * sVr;   // -j v_j dS/dv_j
                    if (jj[j] == row) {
                        kd = k;
                        dTr = sTr;
                        dTi = sTi;
                        dVr = sVr;
                        dVi = sVi;
                    } else {
                        const int p = 2 * rs + k;
                        J[p] = sTr;
                        J[p + d] = sVr;
                        J[2 * nnz + p] = sTi;
                        J[2 * nnz + p + d] = sVi;
                    }
                } else {
                    const double Vjr = vj[j] * c, Vji = vj[j] * s;
                    Ir = fma(yy[j].x, Vjr, Ir);
                    Ir = fma(-yy[j].y, Vji, Ir);
                    Ii = fma(yy[j].x, Vji, Ii);
                    Ii = fma(yy[j].y, Vjr, Ii);
                }
            }
        }
    }
#pragma unroll
    for (int off = W / 2; off > 0; off >>= 1) {
        Ir += __shfl_xor_sync(0xffffffffu, Ir, off, W);
        Ii += __shfl_xor_sync(0xffffffffu, Ii, off, W);
    }
    if (!valid) return;
    const double Sr = fma(Vr, Ir, Vi * Ii), Si = fma(Vi, Ir, -Vr * Ii);
    if (JAC && kd >= 0) {
        dTr -= Si;                        // + j S_i
        dTi += Sr;
        dVr += fma(Ir, cs, Ii * si);      // + conj(I_i) U_i
        dVi += fma(Ir, si, -Ii * cs);
        const int p = 2 * rs + kd;
        J[p] = dTr;
        J[p + d] = dVr;
        J[2 * nnz + p] = dTi;
        J[2 * nnz + p + d] = dVi;
    }
    if (lane == 0 && P) {
        P[row] = Sr;
        Q[row] = Si;
    }
}

template <int W, bool JAC>
static cudaError_t fused_w(const Grid *g, const double *vm, const double *va, double *P, double *Q, double *J,
                           cudaStream_t s)
{
    const long long threads = (long long)g->nb * W;
    const int blk = g->cfg.ybus_block;
    return launch_k(k_ybus_fused<W, JAC>, (int)((threads + blk - 1) / blk), blk, 0, s, true, g->nb, g->nnz,
                    (const int *)g->yrow, (const int *)g->rp, (const int *)g->ci, (const double2 *)g->yv, vm, va, trig_table(), P, Q, J);
}

cudaError_t launch_ybus_fused(const Grid *g, bool jac, const double *vm, const double *va, double *P, double *Q,
                              double *J, cudaStream_t s)
{
    switch (g->cfg.ybus_lanes) {
    case 1: return jac ? fused_w<1, true>(g, vm, va, P, Q, J, s) : fused_w<1, false>(g, vm, va, P, Q, J, s);
    case 2: return jac ? fused_w<2, true>(g, vm, va, P, Q, J, s) : fused_w<2, false>(g, vm, va, P, Q, J, s);
    case 4: return jac ? fused_w<4, true>(g, vm, va, P, Q, J, s) : fused_w<4, false>(g, vm, va, P, Q, J, s);
    case 8: return jac ? fused_w<8, true>(g, vm, va, P, Q, J, s) : fused_w<8, false>(g, vm, va, P, Q, J, s);
    case 16: return jac ? fused_w<16, true>(g, vm, va, P, Q, J, s) : fused_w<16, false>(g, vm, va, P, Q, J, s);
    default: return jac ? fused_w<32, true>(g, vm, va, P, Q, J, s) : fused_w<32, false>(g, vm, va, P, Q, J, s);
    }
}

template <int W>
static cudaError_t inj_w(const Grid *g, const double2 *V, double *P, double *Q, cudaStream_t s)
{
    const long long threads = (long long)g->nb * W;
    const int blk = g->cfg.ybus_block;
    return launch_k(k_inj_ybus<W>, (int)((threads + blk - 1) / blk), blk, 0, s, true, g->nb, (const int *)g->yrow,
                    (const int *)g->rp,
                    (const int *)g->ci, (const double2 *)g->yv, V, P, Q);
}

template <int W>
static cudaError_t jac_w(const Grid *g, const double4_32a *U, double *P, double *Q, double *J, cudaStream_t s)
{
    const long long threads = (long long)g->nb * W;
    const int blk = g->cfg.ybus_block;
    return launch_k(k_jac_ybus<W>, (int)((threads + blk - 1) / blk), blk, 0, s, true, g->nb, g->nnz,
                    (const int *)g->yrow, (const int *)g->rp, (const int *)g->ci, (const double2 *)g->yv, U, P, Q, J);
}

cudaError_t launch_inj_ybus(const Grid *g, const double2 *V, double *P, double *Q, cudaStream_t s)
{
    switch (g->cfg.ybus_lanes) {
    case 1: return inj_w<1>(g, V, P, Q, s);
    case 2: return inj_w<2>(g, V, P, Q, s);
    case 4: return inj_w<4>(g, V, P, Q, s);
    case 8: return inj_w<8>(g, V, P, Q, s);
    case 16: return inj_w<16>(g, V, P, Q, s);
    default: return inj_w<32>(g, V, P, Q, s);
    }
}

cudaError_t launch_jac_ybus(const Grid *g, const double4_32a *U, double *P, double *Q, double *J, cudaStream_t s)
{
    switch (g->cfg.ybus_lanes) {
    case 1: return jac_w<1>(g, U, P, Q, J, s);
    case 2: return jac_w<2>(g, U, P, Q, J, s);
    case 4: return jac_w<4>(g, U, P, Q, J, s);
    case 8: return jac_w<8>(g, U, P, Q, J, s);
    case 16: return jac_w<16>(g, U, P, Q, J, s);
    default: return jac_w<32>(g, U, P, Q, J, s);
    }
}

}  // namespace pf
