// k_ybus_batched.cu - Ybus method (Sec. II-A, IV-B) over a batch of
// scenarios, each of which may lose one branch (an N-1 contingency).
//
// The base CSR Ybus is shared; scenario s's admittance matrix differs from
// it only in the rows of the outage branch's two end buses h and k: the
// branch's terminal constants are taken out of the diagonal entries
// (Y_hh - Ys_h, Y_kk - Ys_k) and of the coupling entries (Y_hk - Yc_h,
// Y_kh - Yc_k), and unless a parallel branch keeps it, the coupling pair
// leaves the pattern altogether.  So W lanes per (scenario, row) run the
// single-scenario kernels of k_ybus.cu with those corrections applied on the
// fly, and write the Jacobian compacted onto scenario s's own pattern at
// J + joff[s] (the closed form of k_batched.cu):
//   rowptr_s[i] = rowptr[i] - del ([h < i] + [k < i]),  d_s(i) = d(i) - del [i in {h, k}],
//   k_s = k - del [k > position of the removed entry in row i].
// Phasors of all scenarios come first, from the flat phasor kernel, in the
// fixed-point form (2^62-scaled cosine and sine); the complex products of the
// base entries run in fixed point on the integer pipe as in k_ybus_fused, the
// entries an outage changes (and values the fixed-point form does not hold)
// in FP64.
#include "fixrot.cuh"
#include "pf_internal.h"
#include "ptx.cuh"

namespace pf {

// entries per lane prefetched together (measured: the batched kernels run
// faster with 4 for every W, although that costs registers)
template <int W>
constexpr int kChunkBW = 4;

// Per-row view of the scenario's outage: the base position of the outage
// branch's entry in this row (-1 if the row is not an outage end) and the
// constants to take out of it and of the diagonal.
struct RowOutage {
    int kx, del;
    double2 dself, dcoup;
};

__device__ __forceinline__ RowOutage row_outage(const ScenOut &o, int i, const double2 *tself,
                                                const double2 *tcoup)
{
    RowOutage r{-1, o.del, make_double2(0.0, 0.0), make_double2(0.0, 0.0)};
    const int p = i == o.h ? o.ph : (i == o.k ? o.pk : -1);
    if (p >= 0) {
        r.kx = i == o.h ? o.kh : o.kk;
        r.dself = tself[p];
        r.dcoup = tcoup[p];
    }
    return r;
}

// Y value of base entry (k, column j) of row i in the scenario; false if the
// entry has left the scenario's pattern.
__device__ __forceinline__ bool scen_value(const RowOutage &r, int i, int k, int j, double2 &y)
{
    if (k == r.kx) {
        if (r.del) return false;
        y.x -= r.dcoup.x;
        y.y -= r.dcoup.y;
    } else if (j == i && r.kx >= 0) {
        y.x -= r.dself.x;
        y.y -= r.dself.y;
    }
    return true;
}

// U[x] = {2^62 cos, 2^62 sin (64-bit integers stored bit for bit), v, -}
__device__ __forceinline__ void unpack_u(const double4_32a &u, int64_t *C, int64_t *S)
{
    *C = __double_as_longlong(u.x);
    *S = __double_as_longlong(u.y);
}

// Y_ij U_j of base entry k (column j) of row i in the scenario, in fixed point
// unless the outage changes the entry; false if the entry has left the
// scenario's pattern.  The changed entries and the values the fixed-point form
// does not hold: FP64 products.
__device__ __forceinline__ bool scen_yu(const RowOutage &ro, int i, int k, int j, const double2 *Y, long long e,
                                        const longlong2 &yf, int ye, int64_t C, int64_t S, double *yur, double *yui)
{
    if (k == ro.kx && ro.del) return false;
    const bool changed = k == ro.kx || (j == i && ro.kx >= 0);
    if (!changed && ye != 0 && C != kFixNaN) {
        fix_ybus_yu(yf.x, yf.y, ye, C, S, yur, yui);
        return true;
    }
    double2 y = Y[e];
    scen_value(ro, i, k, j, y);
    const double c = fix_q62_or_nan(C), s = C == kFixNaN ? c : q62_to_double(S);
    *yur = fma(y.x, c, -y.y * s);
    *yui = fma(y.x, s, y.y * c);
    return true;
}

template <int W, bool OUT>
__global__ void __launch_bounds__(512) k_inj_ybus_b(int S, int nb, const int *__restrict__ yrow,
                                                     const int *__restrict__ rp,
                                                     const int *__restrict__ ci, const double2 *__restrict__ Y,
                                                     const longlong2 *__restrict__ Yf, const int *__restrict__ Ye,
                                                     const double2 *__restrict__ tself,
                                                     const double2 *__restrict__ tcoup,
                                                     const ScenOut *__restrict__ sc, const double4_32a *__restrict__ U,
                                                     double *__restrict__ P, double *__restrict__ Q)
{
    pdl_launch_dependents();   // the next phasor launch may start (it waits for this grid)
    const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long row = gid / W;
    const int lane = (int)(gid % W);
    const bool valid = row < (long long)S * nb;
    // rows of each chunk by decreasing length (Grid::yrow)
    const int s = valid ? (int)(row / nb) : 0, i = valid ? yrow[(int)(row % nb)] : 0;
    int rs = 0, d = 0;
    int jj[kChunkBW<W>];
    longlong2 yf[kChunkBW<W>];
    int ye[kChunkBW<W>];
    if (valid) {
        rs = rp[i];
        d = rp[i + 1] - rs;
    }
#pragma unroll
    for (int j = 0; j < kChunkBW<W>; ++j) {
        const int k = lane + W * j;
        if (k < d) {
            jj[j] = ci[rs + k];
            prefetch_l2(Yf + rs + k);   // parameter data: into L2 before the wait, read after it
            prefetch_l2(Ye + rs + k);
        }
    }
    pdl_wait();
#pragma unroll
    for (int j = 0; j < kChunkBW<W>; ++j) {
        const int k = lane + W * j;
        if (k < d) {   // parameter-dependent (as the outage's constants): after the wait
            yf[j] = Yf[rs + k];
            ye[j] = Ye[rs + k];
        }
    }
    RowOutage ro{-1, 0, make_double2(0.0, 0.0), make_double2(0.0, 0.0)};
    if (OUT && valid) ro = row_outage(sc[s], i, tself, tcoup);
    const double4_32a *Us = U + (long long)s * nb;
    double Ir = 0.0, Ii = 0.0;
    for (int k0 = lane; k0 < d; k0 += W * kChunkBW<W>) {
        if (k0 != lane) {
#pragma unroll
            for (int j = 0; j < kChunkBW<W>; ++j) {
                const int k = k0 + W * j;
                if (k < d) {
                    jj[j] = ci[rs + k];
                    yf[j] = Yf[rs + k];
                    ye[j] = Ye[rs + k];
                }
            }
        }
        double4_32a uu[kChunkBW<W>];
#pragma unroll
        for (int j = 0; j < kChunkBW<W>; ++j)
            if (k0 + W * j < d) uu[j] = Us[jj[j]];
#pragma unroll
        for (int j = 0; j < kChunkBW<W>; ++j) {
            const int k = k0 + W * j;
            if (k < d) {
                int64_t C, Sn;
                unpack_u(uu[j], &C, &Sn);
                double YUr, YUi;
                if (scen_yu(ro, i, k, jj[j], Y, rs + k, yf[j], ye[j], C, Sn, &YUr, &YUi)) {
                    Ir = fma(uu[j].z, YUr, Ir);   // I_i += Y_ij V_j
                    Ii = fma(uu[j].z, YUi, Ii);
                }
            }
        }
    }
#pragma unroll
    for (int off = W / 2; off > 0; off >>= 1) {
        Ir += __shfl_xor_sync(0xffffffffu, Ir, off, W);
        Ii += __shfl_xor_sync(0xffffffffu, Ii, off, W);
    }
    if (valid && lane == 0) {
        const double4_32a ui = Us[i];
        int64_t C, Sn;
        unpack_u(ui, &C, &Sn);
        const double cs = fix_q62_or_nan(C), sn = C == kFixNaN ? cs : q62_to_double(Sn);
        const double Vr = ui.z * cs, Vi = ui.z * sn;
        P[(long long)s * nb + i] = fma(Vr, Ir, Vi * Ii);   // S = V conj(I)
        Q[(long long)s * nb + i] = fma(Vi, Ir, -Vr * Ii);
    }
}

template <int W, bool OUT>
__global__ void __launch_bounds__(512) k_jac_ybus_b(int S, int nb, int nnz, const int *__restrict__ yrow,
                                                     const int *__restrict__ rp,
                                                     const int *__restrict__ ci, const double2 *__restrict__ Y,
                                                     const longlong2 *__restrict__ Yf, const int *__restrict__ Ye,
                                                     const double2 *__restrict__ tself,
                                                     const double2 *__restrict__ tcoup,
                                                     const ScenOut *__restrict__ sc,
                                                     const long long *__restrict__ joff,
                                                     const double4_32a *__restrict__ U, double *__restrict__ P,
                                                     double *__restrict__ Q, double *__restrict__ J)
{
    pdl_launch_dependents();   // the next phasor launch may start (it waits for this grid)
    const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long row = gid / W;
    const int lane = (int)(gid % W);
    const bool valid = row < (long long)S * nb;
    // rows of each chunk by decreasing length (Grid::yrow)
    const int s = valid ? (int)(row / nb) : 0, i = valid ? yrow[(int)(row % nb)] : 0;
    int rs = 0, d = 0;
    int jj[kChunkBW<W>];
    longlong2 yf[kChunkBW<W>];
    int ye[kChunkBW<W>];
    if (valid) {
        rs = rp[i];
        d = rp[i + 1] - rs;
    }
#pragma unroll
    for (int j = 0; j < kChunkBW<W>; ++j) {
        const int k = lane + W * j;
        if (k < d) {
            jj[j] = ci[rs + k];
            prefetch_l2(Yf + rs + k);   // parameter data: into L2 before the wait, read after it
            prefetch_l2(Ye + rs + k);
        }
    }
    // without outages every scenario's Jacobian is the base pattern, 4 nnz values apart
    ScenOut o{-1, -1, -1, -1, 0, 0, 0, -1};
    long long jo = 4LL * nnz * s;
    if (OUT && valid) {
        o = sc[s];
        jo = joff[s];
    }
    pdl_wait();
#pragma unroll
    for (int j = 0; j < kChunkBW<W>; ++j) {
        const int k = lane + W * j;
        if (k < d) {   // parameter-dependent (as the outage's constants): after the wait
            yf[j] = Yf[rs + k];
            ye[j] = Ye[rs + k];
        }
    }
    const RowOutage ro = row_outage(o, i, tself, tcoup);
    // scenario s's compacted row: start, length, and its J halves
    const int del = o.del;
    const int rss = rs - del * ((o.h >= 0 && o.h < i) + (o.k >= 0 && o.k < i));
    const int ds = d - (ro.kx >= 0 ? del : 0);
    const long long nnzs = nnz - 2 * del;
    double *Js = J + jo;
    const double4_32a *Us = U + (long long)s * nb;
    double Ir = 0.0, Ii = 0.0;
    double dTr = 0.0, dTi = 0.0, dVr = 0.0, dVi = 0.0;   // diagonal partials (lane that owns it)
    int kd = -1;
    double4_32a ui = make_double4_32a(0.0, 0.0, 0.0, 0.0);
    if (valid) ui = Us[i];
    int64_t Crow, Srow;
    unpack_u(ui, &Crow, &Srow);
    const double cs = fix_q62_or_nan(Crow), sn = Crow == kFixNaN ? cs : q62_to_double(Srow);
    const double vi = ui.z, Vr = vi * cs, Vi = vi * sn;
    int64_t Ari, Aii;
    fix_phasor(Crow, Srow, vi, &Ari, &Aii);
    for (int k0 = lane; k0 < d; k0 += W * kChunkBW<W>) {
        if (k0 != lane) {
#pragma unroll
            for (int j = 0; j < kChunkBW<W>; ++j) {
                const int k = k0 + W * j;
                if (k < d) {
                    jj[j] = ci[rs + k];
                    yf[j] = Yf[rs + k];
                    ye[j] = Ye[rs + k];
                }
            }
        }
        double4_32a uu[kChunkBW<W>];
#pragma unroll
        for (int j = 0; j < kChunkBW<W>; ++j)
            if (k0 + W * j < d) uu[j] = Us[jj[j]];
#pragma unroll
        for (int j = 0; j < kChunkBW<W>; ++j) {
            const int k = k0 + W * j;
            if (k >= d || (k == ro.kx && del)) continue;   // beyond the row, or left the scenario's pattern
            int64_t C, Sn;
            unpack_u(uu[j], &C, &Sn);
            const bool changed = k == ro.kx || (jj[j] == i && ro.kx >= 0);
            double YUr, YUi, sVr, sVi;   // Y_ij U_j and V_i conj(YU)
            if (changed || ye[j] == 0 || C == kFixNaN || Ari == kFixNaN ||
                !fix_ybus_entry(yf[j].x, yf[j].y, ye[j], C, Sn, Ari, Aii, vi, &YUr, &YUi, &sVr, &sVi)) {
                double2 y = Y[rs + k];
                scen_value(ro, i, k, jj[j], y);
                const double c = fix_q62_or_nan(C), sj = C == kFixNaN ? c : q62_to_double(Sn);
                YUr = fma(y.x, c, -y.y * sj);
                YUi = fma(y.x, sj, y.y * c);
                sVr = fma(Vr, YUr, Vi * YUi);
                sVi = fma(Vi, YUr, -Vr * YUi);
            }
            const double vj = uu[j].z;
            Ir = fma(vj, YUr, Ir);
            Ii = fma(vj, YUi, Ii);
            const double sTr = vj * sVi, sTi = -vj * sVr;   // -j v_j dS/dv_j
            const int ks = k - ((del && ro.kx >= 0 && k > ro.kx) ? 1 : 0);
            if (jj[j] == i) {
                kd = ks;
                dTr = sTr;
                dTi = sTi;
                dVr = sVr;
                dVi = sVi;
            } else {
                const long long p = 2LL * rss + ks;
                Js[p] = sTr;
                Js[p + ds] = sVr;
                Js[2 * nnzs + p] = sTi;
                Js[2 * nnzs + p + ds] = sVi;
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
        dVr += fma(Ir, cs, Ii * sn);         // + conj(I_i) U_i
        dVi += fma(Ir, sn, -Ii * cs);
        const long long p = 2LL * rss + kd;
        Js[p] = dTr;
        Js[p + ds] = dVr;
        Js[2 * nnzs + p] = dTi;
        Js[2 * nnzs + p + ds] = dVi;
    }
    if (lane == 0 && P) {
        P[(long long)s * nb + i] = Sr;
        Q[(long long)s * nb + i] = Si;
    }
}

template <int W, bool OUT>
static cudaError_t rows_w(const Grid *g, int S, const ScenOut *sc, const long long *joff, const double4_32a *U,
                          bool jac, double *P, double *Q, double *J, int blk, cudaStream_t s)
{
    const long long threads = (long long)S * g->nb * W;
    const int grid = (int)((threads + blk - 1) / blk);
    if (jac)
        return launch_k(k_jac_ybus_b<W, OUT>, grid, blk, 0, s, true, S, g->nb, g->nnz, (const int *)g->yrow,
                        (const int *)g->rp, (const int *)g->ci, (const double2 *)g->yv, (const longlong2 *)g->yfx,
                        (const int *)g->yce, (const double2 *)g->tself, (const double2 *)g->tcoup, sc, joff, U, P,
                        Q, J);
    return launch_k(k_inj_ybus_b<W, OUT>, grid, blk, 0, s, true, S, g->nb, (const int *)g->yrow,
                    (const int *)g->rp, (const int *)g->ci, (const double2 *)g->yv, (const longlong2 *)g->yfx,
                    (const int *)g->yce, (const double2 *)g->tself, (const double2 *)g->tcoup, sc, U, P, Q);
}

template <bool OUT>
static cudaError_t rows(const Grid *g, int S, const ScenOut *sc, const long long *joff, const double4_32a *U,
                        bool jac, double *P, double *Q, double *J, int lanes, int blk, cudaStream_t s)
{
    switch (lanes) {
    case 1: return rows_w<1, OUT>(g, S, sc, joff, U, jac, P, Q, J, blk, s);
    case 2: return rows_w<2, OUT>(g, S, sc, joff, U, jac, P, Q, J, blk, s);
    case 4: return rows_w<4, OUT>(g, S, sc, joff, U, jac, P, Q, J, blk, s);
    case 8: return rows_w<8, OUT>(g, S, sc, joff, U, jac, P, Q, J, blk, s);
    case 16: return rows_w<16, OUT>(g, S, sc, joff, U, jac, P, Q, J, blk, s);
    default: return rows_w<32, OUT>(g, S, sc, joff, U, jac, P, Q, J, blk, s);
    }
}

// The row kernels over S scenarios from phasors U in the fixed-point form
// (launch_phasor_fix); sc and joff only with outages (out)
cudaError_t launch_ybus_rows(const Grid *g, int S, bool out, const ScenOut *sc, const long long *joff,
                             const double4_32a *U, bool jac, double *P, double *Q, double *J, int lanes, int blk,
                             cudaStream_t s)
{
    if (S == 0 || g->nb == 0) return cudaSuccess;
    return out ? rows<true>(g, S, sc, joff, U, jac, P, Q, J, lanes, blk, s)
               : rows<false>(g, S, sc, joff, U, jac, P, Q, J, lanes, blk, s);
}

cudaError_t launch_ybus_batched(Batch *b, bool jac, const double *vm, const double *va, double *P, double *Q,
                                double *J, cudaStream_t s)
{
    const Grid *g = b->g;
    if (b->S == 0 || g->nb == 0) return cudaSuccess;
    cudaError_t e = launch_phasor_fix(b->S * g->nb, vm, va, b->U, s);
    if (e != cudaSuccess) return e;
    return launch_ybus_rows(g, b->S, b->has_outage, b->sc, b->joff, b->U, jac, P, Q, J, b->cfg.ybus_lanes,
                            b->cfg.ybus_block, s);
}

}  // namespace pf
