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
// Phasors of all scenarios come first, from the flat phasor kernel.
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

template <int W>
__global__ void __launch_bounds__(512) k_inj_ybus_b(int S, int nb, const int *__restrict__ yrow,
                                                     const int *__restrict__ rp,
                                                     const int *__restrict__ ci, const double2 *__restrict__ Y,
                                                     const double2 *__restrict__ tself,
                                                     const double2 *__restrict__ tcoup,
                                                     const ScenOut *__restrict__ sc, const double2 *__restrict__ V,
                                                     double *__restrict__ P, double *__restrict__ Q)
{
    const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long row = gid / W;
    const int lane = (int)(gid % W);
    const bool valid = row < (long long)S * nb;
    // rows of each chunk by decreasing length (Grid::yrow)
    const int s = valid ? (int)(row / nb) : 0, i = valid ? yrow[(int)(row % nb)] : 0;
    int rs = 0, d = 0;
    int jj[kChunkBW<W>];
    double2 yy[kChunkBW<W>];
    if (valid) {
        rs = rp[i];
        d = rp[i + 1] - rs;
    }
#pragma unroll
    for (int j = 0; j < kChunkBW<W>; ++j) {
        const int k = lane + W * j;
        if (k < d) jj[j] = ci[rs + k];
    }
    pdl_wait();
#pragma unroll
    for (int j = 0; j < kChunkBW<W>; ++j) {
        const int k = lane + W * j;
        if (k < d) yy[j] = Y[rs + k];   // parameter-dependent (as the outage's constants): after the wait
    }
    RowOutage ro{-1, 0, make_double2(0.0, 0.0), make_double2(0.0, 0.0)};
    if (valid) ro = row_outage(sc[s], i, tself, tcoup);
    const double2 *Vs = V + (long long)s * nb;
    double Ir = 0.0, Ii = 0.0;
    for (int k0 = lane; k0 < d; k0 += W * kChunkBW<W>) {
        if (k0 != lane) {
#pragma unroll
            for (int j = 0; j < kChunkBW<W>; ++j) {
                const int k = k0 + W * j;
                if (k < d) {
                    jj[j] = ci[rs + k];
                    yy[j] = Y[rs + k];
                }
            }
        }
        double2 vv[kChunkBW<W>];
#pragma unroll
        for (int j = 0; j < kChunkBW<W>; ++j)
            if (k0 + W * j < d) vv[j] = Vs[jj[j]];
#pragma unroll
        for (int j = 0; j < kChunkBW<W>; ++j) {
            double2 y = yy[j];
            if (k0 + W * j < d && scen_value(ro, i, k0 + W * j, jj[j], y)) {
                Ir = fma(y.x, vv[j].x, Ir);
                Ir = fma(-y.y, vv[j].y, Ir);
                Ii = fma(y.x, vv[j].y, Ii);
                Ii = fma(y.y, vv[j].x, Ii);
            }
        }
    }
#pragma unroll
    for (int off = W / 2; off > 0; off >>= 1) {
        Ir += __shfl_xor_sync(0xffffffffu, Ir, off, W);
        Ii += __shfl_xor_sync(0xffffffffu, Ii, off, W);
    }
    if (valid && lane == 0) {
        const double2 Vi = Vs[i];
        P[(long long)s * nb + i] = fma(Vi.x, Ir, Vi.y * Ii);   // S = V conj(I)
        Q[(long long)s * nb + i] = fma(Vi.y, Ir, -Vi.x * Ii);
    }
}

template <int W>
__global__ void __launch_bounds__(512) k_jac_ybus_b(int S, int nb, int nnz, const int *__restrict__ yrow,
                                                     const int *__restrict__ rp,
                                                     const int *__restrict__ ci, const double2 *__restrict__ Y,
                                                     const double2 *__restrict__ tself,
                                                     const double2 *__restrict__ tcoup,
                                                     const ScenOut *__restrict__ sc,
                                                     const long long *__restrict__ joff,
                                                     const double4_32a *__restrict__ U, double *__restrict__ P,
                                                     double *__restrict__ Q, double *__restrict__ J)
{
    const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long row = gid / W;
    const int lane = (int)(gid % W);
    const bool valid = row < (long long)S * nb;
    // rows of each chunk by decreasing length (Grid::yrow)
    const int s = valid ? (int)(row / nb) : 0, i = valid ? yrow[(int)(row % nb)] : 0;
    int rs = 0, d = 0;
    int jj[kChunkBW<W>];
    double2 yy[kChunkBW<W>];
    if (valid) {
        rs = rp[i];
        d = rp[i + 1] - rs;
    }
#pragma unroll
    for (int j = 0; j < kChunkBW<W>; ++j) {
        const int k = lane + W * j;
        if (k < d) jj[j] = ci[rs + k];
    }
    ScenOut o{-1, -1, -1, -1, 0, 0, 0, -1};
    long long jo = 0;
    if (valid) {
        o = sc[s];
        jo = joff[s];
    }
    pdl_wait();
#pragma unroll
    for (int j = 0; j < kChunkBW<W>; ++j) {
        const int k = lane + W * j;
        if (k < d) yy[j] = Y[rs + k];   // parameter-dependent (as the outage's constants): after the wait
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
    const double Vr = ui.z * ui.x, Vi = ui.z * ui.y;
    for (int k0 = lane; k0 < d; k0 += W * kChunkBW<W>) {
        if (k0 != lane) {
#pragma unroll
            for (int j = 0; j < kChunkBW<W>; ++j) {
                const int k = k0 + W * j;
                if (k < d) {
                    jj[j] = ci[rs + k];
                    yy[j] = Y[rs + k];
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
            double2 y = yy[j];
            if (k < d && scen_value(ro, i, k, jj[j], y)) {
                const double YUr = fma(y.x, uu[j].x, -y.y * uu[j].y);
                const double YUi = fma(y.x, uu[j].y, y.y * uu[j].x);
                const double sVr = fma(Vr, YUr, Vi * YUi);    // V_i conj(YU)
                const double sVi = fma(Vi, YUr, -Vr * YUi);
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

template <int W>
static cudaError_t inj_b(const Batch *b, double *P, double *Q, cudaStream_t s)
{
    const Grid *g = b->g;
    const long long threads = (long long)b->S * g->nb * W;
    const int blk = b->cfg.ybus_block;
    return launch_k(k_inj_ybus_b<W>, (int)((threads + blk - 1) / blk), blk, 0, s, true, b->S, g->nb,
                    (const int *)g->yrow,
                    (const int *)g->rp, (const int *)g->ci, (const double2 *)g->yv, (const double2 *)g->tself,
                    (const double2 *)g->tcoup, (const ScenOut *)b->sc, (const double2 *)b->V, P, Q);
}

template <int W>
static cudaError_t jac_b(const Batch *b, double *P, double *Q, double *J, cudaStream_t s)
{
    const Grid *g = b->g;
    const long long threads = (long long)b->S * g->nb * W;
    const int blk = b->cfg.ybus_block;
    return launch_k(k_jac_ybus_b<W>, (int)((threads + blk - 1) / blk), blk, 0, s, true, b->S, g->nb, g->nnz,
                    (const int *)g->yrow,
                    (const int *)g->rp, (const int *)g->ci, (const double2 *)g->yv, (const double2 *)g->tself,
                    (const double2 *)g->tcoup, (const ScenOut *)b->sc, (const long long *)b->joff,
                    (const double4_32a *)b->U, P, Q, J);
}

cudaError_t launch_ybus_batched(Batch *b, bool jac, const double *vm, const double *va, double *P, double *Q,
                                double *J, cudaStream_t s)
{
    const Grid *g = b->g;
    if (b->S == 0 || g->nb == 0) return cudaSuccess;
    cudaError_t e = launch_phasor(b->S * g->nb, vm, va, b->U, b->V, s);
    if (e != cudaSuccess) return e;
    if (jac) {
        switch (b->cfg.ybus_lanes) {
        case 1: return jac_b<1>(b, P, Q, J, s);
        case 2: return jac_b<2>(b, P, Q, J, s);
        case 4: return jac_b<4>(b, P, Q, J, s);
        case 8: return jac_b<8>(b, P, Q, J, s);
        case 16: return jac_b<16>(b, P, Q, J, s);
        default: return jac_b<32>(b, P, Q, J, s);
        }
    }
    switch (b->cfg.ybus_lanes) {
    case 1: return inj_b<1>(b, P, Q, s);
    case 2: return inj_b<2>(b, P, Q, s);
    case 4: return inj_b<4>(b, P, Q, s);
    case 8: return inj_b<8>(b, P, Q, s);
    case 16: return inj_b<16>(b, P, Q, s);
    default: return inj_b<32>(b, P, Q, s);
    }
}

}  // namespace pf
