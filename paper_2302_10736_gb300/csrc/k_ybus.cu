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
// Two forms: the paper's step 1 as its own launch (k_phasor_fix writes the
// fixed-point phasors of every bus once, and the row kernels of
// k_ybus_batched.cu gather them, as for a batch of one scenario without
// outage), or fused (k_ybus_fused: each lane forms the phasors of its entries'
// columns from vm, va itself, with the integer-pipe sine/cosine of
// isincos.cuh, so one launch evaluates and nothing goes through memory in
// between; a bus's phasor is formed once per entry of its column, about 3.5
// times on these grids).  The autotuner picks the form.
#include "fastmath.cuh"
#include "fixrot.cuh"
#include "pf_internal.h"
#include "ptx.cuh"

namespace pf {

// entries per lane prefetched together: a row of the synthetic grids has about 3.5
// entries, so wide rows (W >= 4 lanes) hold one each and narrow ones several
template <int W>
constexpr int kChunkW = W >= 4 ? 1 : (W == 2 ? 2 : 4);

// Injections (JAC = false) or injections and Jacobian (JAC = true) with the
// phasor step fused: W lanes per row, each forming U_j = e^{j theta_j}, v_j for
// its entries and the row's own V_i.  With the Jacobian the complex products
// Y_ij U_j and V_i conj(Y_ij U_j) run in 64-bit fixed point on the integer
// pipe (fixrot.cuh, from the 2^62-scaled sine and cosine and the setup's
// block-floating Ybus values), the sums I_i = sum_j v_j (Y_ij U_j),
// S_i = V_i conj(I_i) and the Jacobian scalings by v_j in FP64 (values the
// fixed-point form does not hold take FP64 products); the injections alone
// take FP64 products.
template <int W, bool JAC>
__global__ void __launch_bounds__(512) k_ybus_fused(int nb, int nnz, const int *__restrict__ yrow,
                                                     const int *__restrict__ rp,
                                                     const int *__restrict__ ci, const double2 *__restrict__ Y,
                                                     const longlong2 *__restrict__ Yf, const int *__restrict__ Ye,
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
    // the state and the Ybus values may be the previous kernel's: their lines
    // are only brought into L2 before the wait (prefetches return no data)
    if (valid) {
        prefetch_l2(va + row);
        prefetch_l2(vm + row);
    }
#pragma unroll
    for (int j = 0; j < kChunkW<W>; ++j) {
        const int k = lane + W * j;
        if (k < d) {
            prefetch_l2(va + jj[j]);
            prefetch_l2(vm + jj[j]);
            if (JAC) {
                prefetch_l2(Yf + rs + k);
                prefetch_l2(Ye + rs + k);
            } else {
                prefetch_l2(Y + rs + k);
            }
        }
    }
    pdl_wait();
    // the Jacobian takes the block-floating values, the injections the doubles
    longlong2 yf[kChunkW<W>];
    int ye[kChunkW<W>];
    double2 yy[kChunkW<W>];
#pragma unroll
    for (int j = 0; j < kChunkW<W>; ++j) {
        const int k = lane + W * j;
        if (k < d) {
            if (JAC) {
                yf[j] = Yf[rs + k];
                ye[j] = Ye[rs + k];
            } else {
                yy[j] = Y[rs + k];
            }
        }
    }
    const double thi = valid ? va[row] : 0.0, vi = valid ? vm[row] : 0.0;
    __syncthreads();   // the table
    int64_t Crow, Srow;   // 2^62 (cos, sin) of the row's own angle
    int_sincos_q62(thi, tab, &Crow, &Srow);
    const double cs = fix_q62_or_nan(Crow), si = Crow == kFixNaN ? cs : q62_to_double(Srow);
    const double Vr = vi * cs, Vi = vi * si;
    int64_t Ari = kFixNaN, Aii = 0;
    if (JAC) fix_phasor(Crow, Srow, vi, &Ari, &Aii);
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
                    if (JAC) {
                        yf[j] = Yf[rs + k];
                        ye[j] = Ye[rs + k];
                    } else {
                        yy[j] = Y[rs + k];
                    }
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
            if (k < d && JAC) {
                int64_t C, S;
                int_sincos_q62(thj[j], tab, &C, &S);
                double YUr, YUi;   // Y_ij U_j
                {
                    double sVr, sVi;   // V_i conj(YU)
                    if (ye[j] == 0 || C == kFixNaN || Ari == kFixNaN ||
                        !fix_ybus_entry(yf[j].x, yf[j].y, ye[j], C, S, Ari, Aii, vi, &YUr, &YUi, &sVr, &sVi)) {
                        const double2 y = Y[rs + k];
                        const double c = fix_q62_or_nan(C), s = C == kFixNaN ? c : q62_to_double(S);
                        YUr = fma(y.x, c, -y.y * s);
                        YUi = fma(y.x, s, y.y * c);
                        sVr = fma(Vr, YUr, Vi * YUi);
                        sVi = fma(Vi, YUr, -Vr * YUi);
                    }
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
                }
            } else if (k < d) {
                // the injections alone: I_i += Y_ij V_j by FP64 products (the
                // per-entry sine and cosine already load the integer pipe)
                double s, c;
                int_sincos(thj[j], tab, &s, &c);
                const double Vjr = vj[j] * c, Vji = vj[j] * s;
                Ir = fma(yy[j].x, Vjr, Ir);
                Ir = fma(-yy[j].y, Vji, Ir);
                Ii = fma(yy[j].x, Vji, Ii);
                Ii = fma(yy[j].y, Vjr, Ii);
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
                    (const int *)g->yrow, (const int *)g->rp, (const int *)g->ci, (const double2 *)g->yv,
                    (const longlong2 *)g->yfx, (const int *)g->yce, vm, va, trig_table(), P, Q, J);
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

}  // namespace pf
