// k_batched.cu - element-wise method over many scenarios in one persistent
// cooperative launch: N-1 contingency batches and the adjoint of the mismatch
// loss.  (The paper evaluates one state of one grid; batching and
// differentiation are the two extensions this library adds around the same
// per-terminal evaluation and reduction, see k_elementwise.cu.)
//
// Work items are (scenario, window) pairs in scenario-major order, handed to
// the resident CTAs round-robin, so the CTAs active at any time share a few
// scenarios' phasors in L2.  Phase 1 forms every scenario's phasors (flat
// chunks of blockDim.x buses, every lane busy); a grid barrier follows; phase
// 2 evaluates.  The adjoint (k_adj) adds a residual phase and a second
// barrier.  A small batch (about one item per SM) runs k_adj1 instead: one
// item per CTA, each window's own and ghost phasors formed inside the residual
// phase (as k_elementwise.cu does), one grid barrier, and everything the
// gradient phase needs kept in shared memory across it.
//
// Scenario s may remove one branch (outage).  Its two terminals are masked
// (they contribute nothing) and the self sums of its end buses lose the
// branch's self constants.  Unless a parallel branch keeps it, the Ybus entry
// pair (h, k), (k, h) disappears from scenario s's pattern; the Jacobian of
// scenario s is stored compacted on its own pattern at J + joff[s]: with
// del = 1 if the pair disappears, a base slot (row i, position k) moves to
//   rowptr_s[i] = rowptr[i] - del ([h < i] + [k < i]),  d_s(i) = d(i) - del [i in {h, k}],
//   k_s = k - del [(i == h and k > pos(h, k)) or (i == k and k > pos(k, h))],
// the canonical closed form of the scenario's own pattern.
//
// Adjoint (loss L_s = sum_i wP (P_i - Ps_i)^2 + wQ (Q_i - Qs_i)^2, residual
// r_i = (2 wP dP_i, 2 wQ dQ_i), <r, z> = r_P Re z + r_Q Im z):
//   dL/dtheta_q = sum over q's terminals t (other bus o, mirror terminal m):
//                 <r_q, j K_t> + <r_o, -j K_m>
//   dL/dv_q     = <r_q, 2 v_q conj(Yd_q)> + (sum_t <r_q, K_t> + <r_o, K_m>) / v_q
// with K_t = conj(Yc_t) V_q conj(V_o), K_m = conj(Yc_m) V_o conj(V_q): each bus
// sums over its own terminals only (no scatter, fixed order).  Branch
// parameter gradients come from the partials of Eqs. (5)-(6) by g, b, b_sh and
// the tap, one thread per branch summing the scenarios in ascending order.
#include "fastmath.cuh"
#include "fixrot.cuh"
#include "pf_internal.h"
#include "ptx.cuh"

namespace pf {

constexpr uint64_t kBatchBarrierNs = 2000000000ull;   // bounded grid-barrier wait (2 s)

struct BatchArgs {
    int S, nb, nl, nnz, nwin, max_nbus, max_nt, max_L, aligned;
    int max_nph, max_nbr;
    const int *win_bus, *tp, *rp, *kd, *town, *tmir, *tpos, *slotbus, *rorder;
    const int2 *tloc, *brl;
    const int4 *desc;
    const int2 *tnbr;
    const double2 *yd, *tself, *tcoup;
    const longlong2 *tcfx;
    const int *tce;
    const ITrig *trig;
    const ScenOut *sc;
    const long long *joff;
    const double *vm, *va;
    double4_32a *U;
    double2 *V;
    double *P, *Q, *J;
    unsigned int *bar;
    int *err;
    // adjoint
    const double *Ps, *Qs, *wP, *wQ;
    double2 *r;
    double *lpart, *L, *gvm, *gva, *gg, *gb, *gbsh, *gtap;
    const double *Lbar;      // upstream gradient (device scalar; NULL = 1): scales every gradient
    double *Ltot;            // sum_s L_s (may be NULL)
    unsigned int *lcnt;      // scenarios whose L_s is written (the total's arrival count)
    const double *pg, *pb, *pbsh, *ptap, *pshift;
    const int2 *br_hk;
    const double4_32a *br_aux;
};

__device__ __forceinline__ void store_range_ll(double *x, const double *s, long long b0, long long b1)
{
    const int par = (int)(b0 & 1);
    if (par) x[b0] = s[1];
    const long long ge = b0 + par;
    const long long cm = (b1 - ge) & ~1LL;
    if (cm > 0) bulk_s2g(x + ge, s + 2 * par, 8u * (uint32_t)cm);
    if ((b1 - ge) & 1) x[b1 - 1] = s[b1 - 1 - b0 + par];
}

// V = v (c, s) as doubles from the fixed-point phasor: the block-floating
// value rounded on the integer pipe, or FP64 products where the fixed-point
// form does not hold
__device__ __forceinline__ double2 fix_V_double(int64_t C, int64_t S, double v)
{
    int64_t ar, ai;
    fix_phasor(C, S, v, &ar, &ai);
    if (ar != kFixNaN) {
        const int e1 = fix_vexp(v) + 2;   // V = A 2^(e - 1083)
        return make_double2(fix_to_double(ar, e1), fix_to_double(ai, e1));
    }
    const double c = fix_q62_or_nan(C), s = C == kFixNaN ? c : q62_to_double(S);
    return make_double2(v * c, v * s);
}

// phase 1 of the adjoint: the fixed-point phasors of every scenario as in
// batch_phasors_fix (1/v with the gradients), and V as doubles for the
// branch-parameter gradients; chunks of blockDim.x consecutive buses, so that
// every lane has a bus
__device__ __forceinline__ void batch_phasors_adj(const BatchArgs &a, const ITrig *tab, bool grad)
{
    const int tid = threadIdx.x, TB = blockDim.x;
    const int nchunk = (a.nb + TB - 1) / TB;
    const long long nitem = (long long)a.S * nchunk;
    for (long long it = blockIdx.x; it < nitem; it += gridDim.x) {
        const int s = (int)(it / nchunk), c = (int)(it % nchunk);
        const int o = c * TB + tid;
        if (o < a.nb) {
            const long long x = (long long)s * a.nb + o;
            int64_t C, S;
            int_sincos_q62(a.va[x], tab, &C, &S);
            const double v = a.vm[x];
            a.U[x] = make_double4_32a(__longlong_as_double(C), __longlong_as_double(S), v, grad ? fast_rcp(v) : 0.0);
            if (grad) a.V[x] = fix_V_double(C, S, v);
        }
    }
}

// G = conj(Yc_p) V_o conj(U_q) of terminal p (owner o, other bus q) of the
// scenario whose fixed-point phasors start at U: fixed point on the integer
// pipe where it applies (fixrot.cuh), else FP64 products.  *vq = v_q.
__device__ __forceinline__ void batch_G(const BatchArgs &a, const double4_32a *U, int p, int o, int q, double *gr,
                                        double *gi, double *vq)
{
    const longlong2 yf = a.tcfx[p];
    const int ey = a.tce[p];
    const double4_32a uo = U[o], uq = U[q];
    const int64_t Co = __double_as_longlong(uo.x), So = __double_as_longlong(uo.y);
    const int64_t Cq = __double_as_longlong(uq.x), Sq = __double_as_longlong(uq.y);
    int64_t Ar, Ai;
    fix_phasor(Co, So, uo.z, &Ar, &Ai);
    if (Ar == kFixNaN || Cq == kFixNaN || ey == 0 || !fix_G_fast(Ar, Ai, uo.z, Cq, Sq, yf.x, yf.y, ey, gr, gi)) {
        const double2 yc = a.tcoup[p];
        fix_G(Ar, Ai, uo.z, Co, So, Cq, Sq, 0, 0, 0, yc.x, yc.y, gr, gi);
    }
    *vq = uq.z;
}

// phase 1 of the Jacobian and injection batches: the phasors in the
// fixed-point form of the single evaluation (fixrot.cuh), U[x] = {2^62 cos,
// 2^62 sin (64-bit integers, stored bit for bit), v, 1/v (Jacobian only)}
__device__ __forceinline__ void batch_phasors_fix(const BatchArgs &a, const ITrig *tab, bool jac)
{
    const int tid = threadIdx.x, TB = blockDim.x;
    const int nchunk = (a.nb + TB - 1) / TB;
    const long long nitem = (long long)a.S * nchunk;
    for (long long it = blockIdx.x; it < nitem; it += gridDim.x) {
        const int s = (int)(it / nchunk), c = (int)(it % nchunk);
        const int o = c * TB + tid;
        if (o < a.nb) {
            const long long x = (long long)s * a.nb + o;
            int64_t C, S;
            int_sincos_q62(a.va[x], tab, &C, &S);
            const double v = a.vm[x];
            a.U[x] = make_double4_32a(__longlong_as_double(C), __longlong_as_double(S), v, jac ? fast_rcp(v) : 0.0);
        }
    }
}

// Window metadata of item (s, w) into shared memory, corrected for the
// scenario's outage: {J-slice row offset, row length, diagonal position,
// first terminal} per bus and the self sum Yd without the outage branch.
__device__ __forceinline__ void batch_window_meta(const BatchArgs &a, const ScenOut &sc, int b0, int b1, int t0,
                                                  int4 *sbm, double2 *syd)
{
    const int r0 = a.rp[b0];
    for (int b = threadIdx.x; b < b1 - b0; b += blockDim.x) {
        const int o = b0 + b, rs = a.rp[o], kdo = a.kd[o];
        const int del = sc.del;
        const int shift = 2 * del * ((sc.h >= b0 && sc.h < o) + (sc.k >= b0 && sc.k < o));
        const int d = a.rp[o + 1] - rs - del * ((o == sc.h) + (o == sc.k));
        const int kds = kdo - del * ((o == sc.h && kdo > sc.kh) + (o == sc.k && kdo > sc.kk));
        sbm[b] = make_int4(2 * (rs - r0) - shift, d, kds, a.tp[o] - t0);
        double2 y = a.yd[o];
        if (o == sc.h) {
            y.x -= a.tself[sc.ph].x;
            y.y -= a.tself[sc.ph].y;
        }
        if (o == sc.k) {
            y.x -= a.tself[sc.pk].x;
            y.y -= a.tself[sc.pk].y;
        }
        syd[b] = y;
    }
}

template <bool JAC>
__global__ void __launch_bounds__(256, 4) k_ewb(BatchArgs a)
{
    extern __shared__ __align__(16) char smem[];
    const GridBar gbar = grid_barrier_begin(a.bar);
    const EwSmem sp = ew_smem_plan(a.max_nbus, a.max_nt, JAC ? a.max_L : 0, JAC);
    int4 *sbm = reinterpret_cast<int4 *>(smem + sp.bm);
    double2 *syd = reinterpret_cast<double2 *>(smem + sp.yd);
    double2 *skg = reinterpret_cast<double2 *>(smem + sp.kg);
    int *skp = reinterpret_cast<int *>(smem + sp.kp);
    double *jst = reinterpret_cast<double *>(smem + sp.jst);
    double *spq = reinterpret_cast<double *>(smem + sp.pq);
    ITrig *tab = reinterpret_cast<ITrig *>(smem + sp.total);
    const int tid = threadIdx.x, TB = blockDim.x;
    const ITrig *trig = a.trig + (blockIdx.x % kITrigCopies) * kITrigN;
    for (int k = tid; k < kITrigN; k += TB) tab[k] = trig[k];
    __syncthreads();
    batch_phasors_fix(a, tab, JAC);
    if (!grid_barrier(gbar, a.bar, gridDim.x, 0, a.err, DEV_TIMEOUT, kBatchBarrierNs)) return;

    const long long nitem = (long long)a.S * a.nwin;
    for (long long it = blockIdx.x; it < nitem; it += gridDim.x) {
        const int s = (int)(it / a.nwin), w = (int)(it % a.nwin);
        const ScenOut sc = a.sc[s];
        const int b0 = a.win_bus[w], b1 = a.win_bus[w + 1], nbus = b1 - b0;
        const int t0 = a.tp[b0], nt = a.tp[b1] - t0;
        const int del = sc.del;
        const int ndb = del * ((sc.h >= 0 && sc.h < b0) + (sc.k >= 0 && sc.k < b0));
        const int ndw = del * ((sc.h >= b0 && sc.h < b1) + (sc.k >= b0 && sc.k < b1));
        const int r0s = a.rp[b0] - ndb;
        const int Ls = JAC ? 2 * (a.rp[b1] - a.rp[b0]) - 2 * ndw : 0;
        const int nnzs = a.nnz - 2 * del;
        const long long sb = (long long)s * a.nb;
        __syncthreads();   // previous item's shared-memory readers are done
        batch_window_meta(a, sc, b0, b1, t0, sbm, syd);
        // the reduction thread's bus: the window's buses by decreasing terminal count
        double4_32a ub = make_double4_32a(0.0, 0.0, 0.0, 0.0);
        double vb = 0.0;
        int bo = 0;
        if (tid < nbus) {
            bo = a.rorder[b0 + tid];
            if (JAC)
                ub = a.U[sb + b0 + bo];
            else
                vb = a.vm[sb + b0 + bo];
        }
        __syncthreads();
        for (int i = tid; i < nt; i += TB) {
            const int p = t0 + i;
            const int2 nq = a.tnbr[p];
            const int ol = a.town[p] - b0, o = b0 + ol;
            const bool masked = p == sc.ph || p == sc.pk;
            // G = conj(Yc) V_o conj(U_q) on the integer pipe, as in the single evaluation
            double Gr, Gi, vq;
            batch_G(a, a.U + sb, p, o, nq.x, &Gr, &Gi, &vq);
            if (JAC) {
                if (masked) Gr = Gi = 0.0;
                const double Kr = vq * Gr, Ki = vq * Gi;
                const int kp = nq.y & EW_KMASK;
                const int kps = kp - del * ((o == sc.h && kp > sc.kh) + (o == sc.k && kp > sc.kk));
                const bool gone = del && ((o == sc.h && kp == sc.kh) || (o == sc.k && kp == sc.kk));
                skg[2 * i] = make_double2(Kr, Ki);
                skg[2 * i + 1] = make_double2(Gr, Gi);
                skp[i] = gone ? 0 : (kps | (nq.y & EW_ACCUM));
                if (!gone && !(nq.y & EW_ACCUM)) {
                    const int4 bm = sbm[ol];
                    const int pos = bm.x + kps, d = bm.y;
                    jst[pos] = Ki;
                    jst[pos + d] = Gr;
                    jst[Ls + pos] = neg(Kr);
                    jst[Ls + pos + d] = Gi;
                }
            } else {
                double Kr = vq * Gr, Ki = vq * Gi;
                if (masked) Kr = Ki = 0.0;
                skg[i] = make_double2(Kr, Ki);
            }
        }
        __syncthreads();
        const int pqs = (int)sp.pqs;
        const int par = (int)((sb + b0) & 1);
        for (int x = tid; x < nbus; x += TB) {
            const int b = x == tid ? bo : a.rorder[b0 + x];
            const int4 bm = sbm[b];
            const int tend = b + 1 < nbus ? sbm[b + 1].w : nt;
            const double2 y = syd[b];
            // sums start from the first terminal (never EW_ACCUM: it starts its run)
            double sKr = 0.0, sKi = 0.0;
            int i1 = bm.w;
            if (i1 < tend) {
                const double2 K = skg[JAC ? 2 * i1 : i1];
                sKr = K.x;
                sKi = K.y;
                ++i1;
            }
            if (JAC) {
                const int d = bm.y;
                for (int i = i1; i < tend; ++i) {
                    const double2 K = skg[2 * i];
                    sKr += K.x;
                    sKi += K.y;
                    const int kp = skp[i];
                    if (kp & EW_ACCUM) {
                        const double2 G = skg[2 * i + 1];
                        const int pos = bm.x + (kp & EW_KMASK);
                        jst[pos] += K.y;
                        jst[pos + d] += G.x;
                        jst[Ls + pos] -= K.x;
                        jst[Ls + pos + d] += G.y;
                    }
                }
                const double4_32a uo = x == tid ? ub : a.U[sb + b0 + b];
                const double v = uo.z, iv = uo.w, v2 = v * v, tv = fix_twice(v);
                const int pos = bm.x + bm.z;
                // 2 v conj(Yd) + sum K / v and S = v^2 conj(Yd) + sum K, in the
                // single evaluation's order of operations (its products are
                // rounded before the sums: __dmul_rn keeps them from being
                // contracted into FMAs here)
                jst[pos] = neg(sKi);
                jst[pos + d] = fma(sKr, iv, __dmul_rn(tv, y.x));
                jst[Ls + pos] = sKr;
                jst[Ls + pos + d] = fma(sKi, iv, neg(__dmul_rn(tv, y.y)));
                spq[b + par] = sKr + __dmul_rn(v2, y.x);
                spq[pqs + b + par] = sKi + neg(__dmul_rn(v2, y.y));
            } else {
                for (int i = i1; i < tend; ++i) {
                    sKr += skg[i].x;
                    sKi += skg[i].y;
                }
                const double v = x == tid ? vb : a.vm[sb + b0 + b], v2 = v * v;
                spq[b + par] = fma(v2, y.x, sKr);
                spq[pqs + b + par] = fma(-v2, y.y, sKi);
            }
        }
        double *Js = JAC ? a.J + a.joff[s] : nullptr;
        if (a.aligned) {
            fence_proxy_async_smem();
            __syncthreads();
            if (tid == 0) {
                if (JAC) {
                    bulk_s2g(Js + 2 * (long long)r0s, jst, 8u * (uint32_t)Ls);
                    bulk_s2g(Js + 2 * (long long)nnzs + 2 * (long long)r0s, jst + Ls, 8u * (uint32_t)Ls);
                }
                if (a.P) {
                    store_range_ll(a.P, spq, sb + b0, sb + b1);
                    store_range_ll(a.Q, spq + pqs, sb + b0, sb + b1);
                }
                bulk_commit();
                bulk_wait_read();
            }
        } else {
            __syncthreads();
            if (JAC) {
                for (int x = tid; x < Ls; x += TB) {
                    Js[2 * (long long)r0s + x] = jst[x];
                    Js[2 * (long long)nnzs + 2 * (long long)r0s + x] = jst[Ls + x];
                }
            }
            if (a.P)
                for (int b = tid; b < nbus; b += TB) {
                    a.P[sb + b0 + b] = spq[b + par];
                    a.Q[sb + b0 + b] = spq[pqs + b + par];
                }
        }
    }
}

// ------------------------------------------------------------ adjoint ----

// Sum over the 32 lanes of a warp; lane 0's result has a fixed association
// order, so the sums below are the same from run to run.
__device__ __forceinline__ double warp_sum(double x)
{
    for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
    return x;
}

// The loss terms spq[0 .. nbus) of one window, summed by warp 0.
__device__ __forceinline__ void window_loss(const double *spq, int nbus, double *out)
{
    if (threadIdx.x < 32) {
        double acc = 0.0;
        for (int b = threadIdx.x; b < nbus; b += 32) acc += spq[b];
        acc = warp_sum(acc);
        if (threadIdx.x == 0) *out = acc;
    }
}

// The total loss L_total = sum_s L_s (G14), in ascending s by one thread:
// every warp that has written L_s values publishes them and adds their count
// to a.lcnt; the one whose count completes the S scenarios sums them and
// resets the counter for the next launch.  Nothing waits on another CTA.
// Called by lane 0 of the writing warp.
__device__ __forceinline__ void loss_total_arrive(const BatchArgs &a, unsigned int nwritten)
{
    if (!a.Ltot || nwritten == 0) return;
    __threadfence();
    const unsigned int prev = atomicAdd(a.lcnt, nwritten);
    if (prev + nwritten != (unsigned int)a.S) return;
    __threadfence();
    double t = 0.0;
    int s = 0;
    for (; s + 8 <= a.S; s += 8) {
        double x[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) x[u] = __ldcg(a.L + s + u);
#pragma unroll
        for (int u = 0; u < 8; ++u) t += x[u];
    }
    for (; s < a.S; ++s) t += __ldcg(a.L + s);
    *a.Ltot = t;
    *a.lcnt = 0u;
}

// The loss of every scenario from its window partial sums, one warp per
// scenario (after the last grid barrier), then the total.
__device__ __forceinline__ void batch_loss(const BatchArgs &a)
{
    const int lane = threadIdx.x & 31;
    const long long nwarp = ((long long)gridDim.x * blockDim.x) >> 5;
    unsigned int nw = 0;
    for (long long s = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; s < a.S; s += nwarp) {
        double acc = 0.0;
        for (int w = lane; w < a.nwin; w += 32) acc += __ldcg(a.lpart + s * a.nwin + w);
        acc = warp_sum(acc);
        if (lane == 0) a.L[s] = acc;
        ++nw;
    }
    if (lane == 0) loss_total_arrive(a, nw);
}

// Branch-parameter gradients: the partials of Eqs. (5)-(6) by g, b, b_sh and
// the tap m of branch (h, k), paired with the end residuals.  With
// B = V_h conj(V_k) e^{-j phi}, A_h = v_h^2 / m^2, s_x = r_h.x + r_k.x,
// d_x = r_h.x - r_k.x (likewise s_y, d_y), Q1 = B.x s_x + B.y d_y,
// Q2 = B.x s_y - B.y d_x and S_sh = r_h.y A_h + r_k.y v_k^2, one scenario adds
//   dL/dg    += r_h.x A_h + r_k.x v_k^2 - Q1 / m
//   dL/db    += Q2 / m - S_sh
//   dL/db_sh += -S_sh / 2
//   dL/dm    += (-2 A_h (r_h.x g + r_h.y c1i) + (g Q1 - b Q2) / m) / m,  c1i = -(b + b_sh/2).
struct BranchConst {
    int h, k;
    double g, bb, im, cphi, sphi, c1i;
};

__device__ __forceinline__ BranchConst branch_const(const BatchArgs &a, int l)
{
    const int2 hk = a.br_hk[l];
    const double4_32a aux = a.br_aux[l];   // 1/m, cos phi, sin phi, c1i (formed with the constants)
    return BranchConst{hk.x, hk.y, a.pg[l], a.pb[l], aux.x, aux.y, aux.z, aux.w};
}

template <bool ACC>
__device__ __forceinline__ void branch_terms(const BranchConst &c, double2 Vh, double2 Vk, double2 rh, double2 rk,
                                             double &agg, double &agb, double &agsh, double &agt)
{
    const double im = c.im;
    const double vh2 = fma(Vh.x, Vh.x, Vh.y * Vh.y), vk2 = fma(Vk.x, Vk.x, Vk.y * Vk.y);
    const double Wr = fma(Vh.x, Vk.x, Vh.y * Vk.y), Wi = fma(Vh.y, Vk.x, -Vh.x * Vk.y);   // V_h conj(V_k)
    const double Br = fma(Wr, c.cphi, Wi * c.sphi), Bi = fma(Wi, c.cphi, -Wr * c.sphi);   // W e^{-j phi}
    const double sx = rh.x + rk.x, dx = rh.x - rk.x, sy = rh.y + rk.y, dy = rh.y - rk.y;
    const double Q1 = fma(Br, sx, Bi * dy), Q2 = fma(Br, sy, -Bi * dx);
    const double Ah = vh2 * (im * im);
    const double Ssh = fma(rh.y, Ah, rk.y * vk2);
    const double tg = fma(-im, Q1, fma(rh.x, Ah, rk.x * vk2));
    const double tb = fma(im, Q2, -Ssh);
    const double tsh = -0.5 * Ssh;
    const double C = fma(rh.x, c.g, rh.y * c.c1i);
    const double tt = im * fma(-2.0 * Ah, C, im * fma(c.g, Q1, -c.bb * Q2));
    if (ACC) {
        agg += tg;
        agb += tb;
        agsh += tsh;
        agt += tt;
    } else {
        agg = tg;
        agb = tb;
        agsh = tsh;
        agt = tt;
    }
}

// one thread per branch summing the scenarios in ascending order, from the
// phasors V and the residuals r of every scenario in global memory
__device__ __forceinline__ void branch_grad(const BatchArgs &a, int l, const BranchConst &c)
{
    double agg = 0.0, agb = 0.0, agsh = 0.0, agt = 0.0;
    bool first = true;
    for (int s = 0; s < a.S; ++s) {
        if (a.sc[s].l == l) continue;   // removed in this scenario
        const long long sb = (long long)s * a.nb;
        const double2 Vh = a.V[sb + c.h], Vk = a.V[sb + c.k], rh = a.r[sb + c.h], rk = a.r[sb + c.k];
        if (first)
            branch_terms<false>(c, Vh, Vk, rh, rk, agg, agb, agsh, agt);
        else
            branch_terms<true>(c, Vh, Vk, rh, rk, agg, agb, agsh, agt);
        first = false;
    }
    a.gg[l] = agg;
    a.gb[l] = agb;
    a.gbsh[l] = agsh;
    a.gtap[l] = agt;
}

// This CTA's branches: a contiguous range of ceil(nl / gridDim.x), so that
// every SM gets the same share of the branch-gradient work.
__device__ __forceinline__ int2 cta_branches(const BatchArgs &a)
{
    const int chunk = (a.nl + (int)gridDim.x - 1) / (int)gridDim.x;
    const int lb = min(a.nl, (int)blockIdx.x * chunk);
    return make_int2(lb, min(a.nl, lb + chunk));
}

// Throughput adjoint (many items per CTA): every scenario's phasors, grid
// barrier, injections and residuals, grid barrier, gradients.  GRAD = false:
// the loss alone (phasors, injections, loss terms, the losses).
template <bool GRAD>
__global__ void __launch_bounds__(256, 4) k_adj(BatchArgs a)
{
    extern __shared__ __align__(16) char smem[];
    const GridBar gbar = grid_barrier_begin(a.bar);
    const EwSmem sp = ew_smem_plan(a.max_nbus, a.max_nt, 0, false);
    int4 *sbm = reinterpret_cast<int4 *>(smem + sp.bm);
    double2 *syd = reinterpret_cast<double2 *>(smem + sp.yd);
    double2 *skg = reinterpret_cast<double2 *>(smem + sp.kg);
    double *spq = reinterpret_cast<double *>(smem + sp.pq);
    ITrig *tab = reinterpret_cast<ITrig *>(smem + sp.total);
    const int tid = threadIdx.x, TB = blockDim.x;
    const ITrig *trig = a.trig + (blockIdx.x % kITrigCopies) * kITrigN;
    for (int k = tid; k < kITrigN; k += TB) tab[k] = trig[k];
    __syncthreads();
    // every scenario's phasors first, visible to all CTAs after the barrier
    batch_phasors_adj(a, tab, GRAD);
    // r = 2 Lbar w dS: the upstream gradient scales every gradient below
    const double tl = 2.0 * (a.Lbar ? *a.Lbar : 1.0);
    if (!grid_barrier(gbar, a.bar, gridDim.x, 0, a.err, DEV_TIMEOUT, kBatchBarrierNs)) return;

    const long long nitem = (long long)a.S * a.nwin;
    // ---- phase 2: injections, residuals and per-window loss partial sums ----
    for (long long it = blockIdx.x; it < nitem; it += gridDim.x) {
        const int s = (int)(it / a.nwin), w = (int)(it % a.nwin);
        const ScenOut sc = a.sc[s];
        const int b0 = a.win_bus[w], b1 = a.win_bus[w + 1], nbus = b1 - b0;
        const int t0 = a.tp[b0], nt = a.tp[b1] - t0;
        const long long sb = (long long)s * a.nb;
        const int bo = tid < nbus ? a.rorder[b0 + tid] : 0;   // by decreasing terminal count
        __syncthreads();
        batch_window_meta(a, sc, b0, b1, t0, sbm, syd);
        for (int i = tid; i < nt; i += TB) {
            const int p = t0 + i;
            double Gr, Gi, vq;   // K_t = v_q G, G = conj(Yc) V_o conj(U_q)
            batch_G(a, a.U + sb, p, a.town[p], a.tnbr[p].x, &Gr, &Gi, &vq);
            double Kr = vq * Gr, Ki = vq * Gi;
            if (p == sc.ph || p == sc.pk) Kr = Ki = 0.0;
            skg[i] = make_double2(Kr, Ki);
        }
        __syncthreads();
        for (int x = tid; x < nbus; x += TB) {
            const int b = x == tid ? bo : a.rorder[b0 + x];
            const int4 bm = sbm[b];
            const int tend = b + 1 < nbus ? sbm[b + 1].w : nt;
            double sKr = 0.0, sKi = 0.0;
            int i = bm.w;
            if (i < tend) {
                sKr = skg[i].x;
                sKi = skg[i].y;
                ++i;
            }
            for (; i < tend; ++i) {
                sKr += skg[i].x;
                sKi += skg[i].y;
            }
            const int o = b0 + b;
            const double v = a.vm[sb + o], v2 = v * v;
            const double2 y = syd[b];
            const double dP = fma(v2, y.x, sKr) - a.Ps[o];
            const double dQ = fma(-v2, y.y, sKi) - a.Qs[o];
            const double wp = a.wP[o], wq = a.wQ[o];
            if (GRAD) a.r[sb + o] = make_double2(tl * wp * dP, tl * wq * dQ);
            spq[x] = fma(wp * dP, dP, wq * dQ * dQ);
        }
        __syncthreads();
        window_loss(spq, nbus, a.lpart + (long long)s * a.nwin + w);
    }
    if (!grid_barrier(gbar, a.bar, gridDim.x, 1, a.err, DEV_TIMEOUT, kBatchBarrierNs)) return;

    // ---- phase 3a: state gradients, one bus per thread over its own terminals ----
    for (long long it = blockIdx.x; GRAD && it < nitem; it += gridDim.x) {
        const int s = (int)(it / a.nwin), w = (int)(it % a.nwin);
        const ScenOut sc = a.sc[s];
        const int b0 = a.win_bus[w], b1 = a.win_bus[w + 1], nbus = b1 - b0;
        const int t0 = a.tp[b0], nt = a.tp[b1] - t0;
        const long long sb = (long long)s * a.nb;
        const int bo = tid < nbus ? a.rorder[b0 + tid] : 0;
        __syncthreads();
        batch_window_meta(a, sc, b0, b1, t0, sbm, syd);
        __syncthreads();
        for (int i = tid; i < nt; i += TB) {
            const int p = t0 + i;
            const int q = a.town[p], o = a.tnbr[p].x;   // q owns the terminal, o is the other end
            const double2 rq = a.r[sb + q], ro = a.r[sb + o];
            // K_t = conj(Yc_t) V_q conj(V_o) = v_o G_t and the mirror's K_m =
            // conj(Yc_m) V_o conj(V_q) = v_q G_m, the G on the integer pipe
            double gtr, gti, gmr, gmi, vo, vq;
            batch_G(a, a.U + sb, p, q, o, &gtr, &gti, &vo);
            batch_G(a, a.U + sb, a.tmir[p], o, q, &gmr, &gmi, &vq);
            const double Kr = vo * gtr, Ki = vo * gti;
            const double Mr = vq * gmr, Mi = vq * gmi;
            double th = fma(-rq.x, Ki, rq.y * Kr) + fma(ro.x, Mi, -ro.y * Mr);
            double vv = fma(rq.x, Kr, rq.y * Ki) + fma(ro.x, Mr, ro.y * Mi);
            if (p == sc.ph || p == sc.pk) th = vv = 0.0;
            skg[i] = make_double2(th, vv);
        }
        __syncthreads();
        const int pqs = (int)sp.pqs;
        const int par = (int)((sb + b0) & 1);
        for (int x = tid; x < nbus; x += TB) {
            const int b = x == tid ? bo : a.rorder[b0 + x];
            const int4 bm = sbm[b];
            const int tend = b + 1 < nbus ? sbm[b + 1].w : nt;
            double gth = 0.0, gv = 0.0;
            int i = bm.w;
            if (i < tend) {
                gth = skg[i].x;
                gv = skg[i].y;
                ++i;
            }
            for (; i < tend; ++i) {
                gth += skg[i].x;
                gv += skg[i].y;
            }
            const int q = b0 + b;
            const double4_32a uq = a.U[sb + q];
            const double2 rq = a.r[sb + q];
            const double2 y = syd[b];
            const double tv = uq.z + uq.z;
            // <r_q, 2 v_q conj(Yd)> + (sum) / v_q
            spq[b + par] = gth;
            spq[pqs + b + par] = fma(gv, uq.w, tv * fma(rq.x, y.x, -rq.y * y.y));
        }
        if (a.aligned) {
            fence_proxy_async_smem();
            __syncthreads();
            if (tid == 0) {
                store_range_ll(a.gva, spq, sb + b0, sb + b1);
                store_range_ll(a.gvm, spq + pqs, sb + b0, sb + b1);
                bulk_commit();
                bulk_wait_read();
            }
        } else {
            __syncthreads();
            for (int b = tid; b < nbus; b += TB) {
                a.gva[sb + b0 + b] = spq[b + par];
                a.gvm[sb + b0 + b] = spq[pqs + b + par];
            }
        }
    }

    // ---- phase 3b: branch-parameter gradients; the loss of every scenario ----
    if (GRAD && a.gg) {
        const int2 lr = cta_branches(a);
        for (int l = lr.x + tid; l < lr.y; l += TB) branch_grad(a, l, branch_const(a, l));
    }
    if (a.L) batch_loss(a);
}

// Small-batch adjoint: one (scenario, window) item per CTA (the launch has a
// CTA for every item) and one grid barrier.  Before the barrier the item
// forms the phasors of its own and ghost buses (slot j's bus in slotbus),
// both flows of every terminal (o owns the terminal): K_t = conj(Yc_t) V_o
// conj(V_q) and the mirror's K_m = conj(Yc_m) V_q conj(V_o), the complex
// products in fixed point on the integer pipe (fixrot.cuh), then its buses'
// injections and residuals.  All of it stays in shared
// memory, so after the barrier the item reads back only its ghost buses'
// residuals (one L2 round trip) before the state gradients (and, for a single
// scenario, the gradients of the branches whose from-terminal it owns)
//   dL/dtheta_o = sum_t <r_o, j K_t> + <r_q, -j K_m>
//   dL/dv_o     = <r_o, 2 v_o conj(Yd_o)> + (sum_t <r_o, K_t> + <r_q, K_m>) / v_o.
// GRAD = false: the loss alone (no mirror flows, residuals or gradients).
template <bool GRAD>
__global__ void __launch_bounds__(kAdj1Threads, 1) k_adj1(BatchArgs a)
{
    extern __shared__ __align__(16) char smem[];
    const GridBar gbar = grid_barrier_begin(a.bar);
    const Adj1Smem sp = adj1_smem_plan(a.max_nbus, a.max_nt, a.max_nph);
    int4 *sbm = reinterpret_cast<int4 *>(smem + sp.bm);
    double2 *syd = reinterpret_cast<double2 *>(smem + sp.yd);
    double2 *sK = reinterpret_cast<double2 *>(smem + sp.K);
    double2 *sM = reinterpret_cast<double2 *>(smem + sp.M);
    int2 *sloc = reinterpret_cast<int2 *>(smem + sp.loc);   // per terminal: {owner slot, other-bus slot}
    __shared__ double swl[32];                                 // per-warp loss partials
    double *spq = reinterpret_cast<double *>(smem + sp.pq);
    double2 *sV = reinterpret_cast<double2 *>(smem + sp.V);
    double2 *sR = reinterpret_cast<double2 *>(smem + sp.R);
    double2 *sW = reinterpret_cast<double2 *>(smem + sp.W);   // own buses: (v, 1/v)
    longlong2 *sUf = reinterpret_cast<longlong2 *>(smem + sp.uf);   // 2^62 (cos, sin)
    longlong2 *sAf = reinterpret_cast<longlong2 *>(smem + sp.af);   // V in block floating point
    double *svs = reinterpret_cast<double *>(smem + sp.vs);         // v
    int *sslot = reinterpret_cast<int *>(smem + sp.slot);
    ITrig *tab = reinterpret_cast<ITrig *>(smem + sp.tab);
    const int tid = threadIdx.x, TB = blockDim.x;
    const bool has = (long long)blockIdx.x < (long long)a.S * a.nwin;   // CTA-uniform
    int s = 0, w = 0, b0 = 0, nbus = 0, t0 = 0, nt = 0, nph = 0;
    long long sb = 0;
    ScenOut sc{};
    // One scenario: each window forms the gradients of the branches whose
    // from-terminal it owns, from its shared-memory phasors and residuals.
    // Several scenarios: a contiguous range of branches per CTA, summing the
    // scenarios from global memory.
    const bool fused = GRAD && a.gg && a.S == 1;
    int nbr = 0;                          // branches of the window (fused)
    int2 e0 = make_int2(0, 0);            // the thread's first: {window-local from-terminal, branch}
    int bo = 0;                           // the bus of the thread's first bus-loop slot
    BranchConst bc0{};
    if (has) {
        s = (int)(blockIdx.x / a.nwin);
        w = (int)(blockIdx.x % a.nwin);
        const int4 d0 = a.desc[2 * w], d1 = a.desc[2 * w + 1];
        b0 = d0.x;
        nbus = d0.y;
        t0 = d0.z;
        nt = d0.w;
        nph = d1.z;
        if (fused) nbr = d1.w;
        sb = (long long)s * a.nb;
        sc = a.sc[s];
        const int *sbus = a.slotbus + (long long)w * a.max_nph;
        // The thread's first phasor slot, terminal and bus are loaded up
        // front, in order of dependence, so that their latency hides behind
        // the window metadata and the phasors.  The sine/cosine table goes
        // with the first level: behind the second-level gathers it would
        // arrive last, and the barrier before the phasors waits for it.
        const int o0 = tid < a.max_nph ? sbus[tid] : 0;
        const ITrig *trig = a.trig + (blockIdx.x % kITrigCopies) * kITrigN;
        ITrig tv0 = {0ull, 0ull};
        if (tid < kITrigN) tv0 = trig[tid];
        longlong2 yf0 = make_longlong2(0, 0), ymf0 = make_longlong2(0, 0);
        int ey0 = 0, eym0 = 0;
        int2 loc0 = make_int2(0, 0);
        int tm0 = 0;
        if (tid < nt) {
            const int p = t0 + tid;
            yf0 = a.tcfx[p];
            ey0 = a.tce[p];
            if (GRAD) tm0 = a.tmir[p];
            loc0 = make_int2(a.town[p], a.tloc[p].x);   // owner made window-local at first use
        }
        if (fused && tid < a.max_nbr) e0 = a.brl[(long long)w * a.max_nbr + tid];
        // two threads per bus below: x = 2b + im, im = 0 the P part, 1 the Q part
        double spec0 = 0.0, wt0 = 0.0;
        if (tid < 2 * nbus) bo = a.rorder[b0 + (tid >> 1)];   // buses by decreasing terminal count
        double th0 = 0.0, v0 = 0.0;
        if (tid < nph) {
            th0 = a.va[sb + o0];
            v0 = a.vm[sb + o0];
        }
        if (tid < kITrigN) tab[tid] = tv0;
        for (int k = tid + TB; k < kITrigN; k += TB) tab[k] = trig[k];
        // nothing before this barrier waits for a second-level load: what
        // depends on one (the bus metadata in shared memory, loads addressed by
        // the reduction order or the mirror terminal) comes after the phasors
        __syncthreads();
        // ---- phasors of the own and ghost buses ----
        for (int j = tid; j < nph; j += TB) {
            int o = o0;
            double th = th0, v = v0;
            if (j != tid) {
                o = sbus[j];
                th = a.va[sb + o];
                v = a.vm[sb + o];
            }
            sslot[j] = o;
            // the fixed-point phasor (fixrot.cuh) and V as doubles (the
            // block-floating value rounded on the integer pipe where it holds)
            int64_t C, S, ar, ai;
            int_sincos_q62(th, tab, &C, &S);
            fix_phasor(C, S, v, &ar, &ai);
            double2 V;
            if (ar != kFixNaN) {
                const int e1 = fix_vexp(v) + 2;   // V = A 2^(e - 1083)
                V = make_double2(fix_to_double(ar, e1), fix_to_double(ai, e1));
            } else {
                const double c = fix_q62_or_nan(C), sn = C == kFixNaN ? c : q62_to_double(S);
                V = make_double2(v * c, v * sn);
            }
            sV[j] = V;
            sUf[j] = make_longlong2(C, S);
            sAf[j] = make_longlong2(ar, ai);
            svs[j] = v;
            if (j < nbus) {
                sW[j] = make_double2(v, GRAD ? fast_rcp(v) : 0.0);
                if (GRAD) a.V[sb + o] = V;   // for the branch-parameter gradients
            }
        }
        batch_window_meta(a, sc, b0, b0 + nbus, t0, sbm, syd);
        if (GRAD && tid < nt) {
            ymf0 = a.tcfx[tm0];
            eym0 = a.tce[tm0];
        }
        if (tid < 2 * nbus) {
            const int o = b0 + bo;
            spec0 = (tid & 1) ? a.Qs[o] : a.Ps[o];
            wt0 = (tid & 1) ? a.wQ[o] : a.wP[o];
        }
        __syncthreads();
        // ---- both flows of every terminal ----
        for (int i = tid; i < nt; i += TB) {
            const int p = t0 + i;
            longlong2 yf = yf0, ymf = ymf0;
            int ey = ey0, eym = eym0, tm = tm0;
            int2 loc = loc0;
            if (i != tid) {
                yf = a.tcfx[p];
                ey = a.tce[p];
                if (GRAD) {
                    tm = a.tmir[p];
                    ymf = a.tcfx[tm];
                    eym = a.tce[tm];
                }
                loc = make_int2(a.town[p], a.tloc[p].x);
            }
            loc.x -= b0;
            // K_t = conj(Yc_t) V_o conj(V_q) = v_q G_t and the mirror's K_m =
            // conj(Yc_m) V_q conj(V_o) = v_o G_m, the G on the integer pipe
            const longlong2 Ao = sAf[loc.x], Uq = sUf[loc.y];
            const double vo = svs[loc.x], vq = svs[loc.y];
            double gr, gi;
            if (Ao.x == kFixNaN || Uq.x == kFixNaN || ey == 0 ||
                !fix_G_fast(Ao.x, Ao.y, vo, Uq.x, Uq.y, yf.x, yf.y, ey, &gr, &gi)) {
                const longlong2 Uo = sUf[loc.x];
                const double2 yc = a.tcoup[p];
                fix_G(Ao.x, Ao.y, vo, Uo.x, Uo.y, Uq.x, Uq.y, 0, 0, 0, yc.x, yc.y, &gr, &gi);
            }
            double Kr = vq * gr, Ki = vq * gi;
            if (p == sc.ph || p == sc.pk) Kr = Ki = 0.0;   // outage branch
            sK[i] = make_double2(Kr, Ki);
            if (GRAD) {
                const longlong2 Aq = sAf[loc.y], Uo = sUf[loc.x];
                double mr, mi;
                if (Aq.x == kFixNaN || Uo.x == kFixNaN || eym == 0 ||
                    !fix_G_fast(Aq.x, Aq.y, vq, Uo.x, Uo.y, ymf.x, ymf.y, eym, &mr, &mi)) {
                    const double2 ym = a.tcoup[tm];
                    fix_G(Aq.x, Aq.y, vq, Uq.x, Uq.y, Uo.x, Uo.y, 0, 0, 0, ym.x, ym.y, &mr, &mi);
                }
                double Mr = vo * mr, Mi = vo * mi;
                if (p == sc.ph || p == sc.pk) Mr = Mi = 0.0;
                sM[i] = make_double2(Mr, Mi);
                sloc[i] = loc;
            }
        }
        __syncthreads();
        // the first branch's constants (not thread 0: its fence on arriving at
        // the barrier would wait for these loads)
        if (fused && tid && tid < nbr) bc0 = branch_const(a, e0.y);
        // ---- injections, residuals and loss terms of the own buses, two
        // threads per bus (the P and the Q part; no divergence) ----
        double lt = 0.0;   // the thread's loss terms
        const double tl = GRAD ? 2.0 * (a.Lbar ? *a.Lbar : 1.0) : 0.0;
        {
            const double *kk = reinterpret_cast<const double *>(sK);
            double *rr = reinterpret_cast<double *>(sR);
            double *gr = reinterpret_cast<double *>(a.r + sb + b0);
            for (int x = tid; x < 2 * nbus; x += TB) {
                const int b = x == tid ? bo : a.rorder[b0 + (x >> 1)], im = x & 1;
                const int4 bm = sbm[b];
                const int tend = b + 1 < nbus ? sbm[b + 1].w : nt;
                int i = bm.w;
                double sk = 0.0;
                if (i < tend) sk = kk[2 * i++ + im];
                for (; i < tend; ++i) sk += kk[2 * i + im];
                double spec = spec0, wt = wt0;
                if (x != tid) {
                    spec = im ? a.Qs[b0 + b] : a.Ps[b0 + b];
                    wt = im ? a.wQ[b0 + b] : a.wP[b0 + b];
                }
                const double v = sW[b].x;
                const double2 y = syd[b];
                // P = v^2 Re conj(Yd) + sum Re K, Q = v^2 Im conj(Yd) + sum Im K
                const double d = fma(v * v, im ? neg(y.y) : y.x, sk) - spec;
                if (GRAD) {
                    const double r = tl * wt * d;   // 2 Lbar w dS
                    gr[2 * b + im] = r;
                    rr[2 * b + im] = r;
                }
                lt = fma(wt * d, d, lt);
            }
        }
        // the window's loss partial: per warp (the warps that hold buses),
        // then over the warps, in a fixed order
        const int lane = tid & 31, wid = tid >> 5, nwb = min(TB >> 5, (2 * nbus + 31) >> 5);
        if (wid < nwb) {
            lt = warp_sum(lt);
            if (lane == 0) swl[wid] = lt;
        }
        __syncthreads();
        if (wid == 0) {
            double x = lane < nwb ? swl[lane] : 0.0;
            x = warp_sum(x);
            if (lane == 0) a.lpart[(long long)s * a.nwin + w] = x;
        }
    }
    // several scenarios: the thread's first branch of the CTA's range
    int2 lr = make_int2(0, 0);
    int l0 = -1;
    if (GRAD && !fused && a.gg) {
        lr = cta_branches(a);
        l0 = lr.x + tid;
        if (tid && l0 < lr.y) bc0 = branch_const(a, l0);
    }
    if (!grid_barrier(gbar, a.bar, gridDim.x, 0, a.err, DEV_TIMEOUT, kBatchBarrierNs)) return;

    const int jg = nbus + tid;
    double2 rg = make_double2(0.0, 0.0);
    if (GRAD && has && jg < nph) rg = a.r[sb + sslot[jg]];
    if (GRAD && tid == 0 && (fused ? tid < nbr : l0 >= 0 && l0 < lr.y)) bc0 = branch_const(a, fused ? e0.y : l0);
    if (GRAD && !fused && a.gg && l0 < lr.y) branch_grad(a, l0, bc0);
    // the loss of scenario blockIdx.x (S <= items <= CTAs), by the last warp,
    // its loads in flight with the ghost residuals'
    if (a.L && blockIdx.x < (unsigned)a.S && (tid >> 5) == (TB >> 5) - 1) {
        const int lane = tid & 31;
        const double *lp = a.lpart + (long long)blockIdx.x * a.nwin;
        double acc = 0.0;
        for (int w2 = lane; w2 < a.nwin; w2 += 32) acc += __ldcg(lp + w2);
        acc = warp_sum(acc);
        if (lane == 0) {
            a.L[blockIdx.x] = acc;
            loss_total_arrive(a, 1u);
        }
    }
    if (GRAD && has) {
        // ---- the ghost buses' residuals ----
        if (jg < nph) sR[jg] = rg;
        for (int j = jg + TB; j < nph; j += TB) sR[j] = a.r[sb + sslot[j]];
        __syncthreads();
        // ---- state-gradient terms of every terminal ----
        for (int i = tid; i < nt; i += TB) {
            const double2 K = sK[i], M = sM[i];
            const int2 loc = sloc[i];
            const double2 ro = sR[loc.x], rq = sR[loc.y];
            const double th = fma(-ro.x, K.y, ro.y * K.x) + fma(rq.x, M.y, -rq.y * M.x);
            const double vv = fma(ro.x, K.x, ro.y * K.y) + fma(rq.x, M.x, rq.y * M.y);
            sK[i] = make_double2(th, vv);
        }
        // the window's branches: h = the from-terminal's owner, k = its other bus
        for (int j = tid; j < nbr; j += TB) {
            int i = e0.x, l = e0.y;
            BranchConst c = bc0;
            if (j != tid) {
                const int2 e = a.brl[(long long)w * a.max_nbr + j];
                i = e.x;
                l = e.y;
                c = branch_const(a, l);
            }
            const int2 loc = sloc[i];
            double agg = 0.0, agb = 0.0, agsh = 0.0, agt = 0.0;
            if (l != sc.l) branch_terms<false>(c, sV[loc.x], sV[loc.y], sR[loc.x], sR[loc.y], agg, agb, agsh, agt);
            a.gg[l] = agg;
            a.gb[l] = agb;
            a.gbsh[l] = agsh;
            a.gtap[l] = agt;
        }
        __syncthreads();
        const int pqs = (int)sp.pqs;
        const int par = (int)((sb + b0) & 1);
        {   // two threads per bus: x = 2b + im sums the theta (im = 0) or v (im = 1) terms
            const double *kk = reinterpret_cast<const double *>(sK);
            for (int x = tid; x < 2 * nbus; x += TB) {
                const int b = x == tid ? bo : a.rorder[b0 + (x >> 1)], im = x & 1;
                const int4 bm = sbm[b];
                const int tend = b + 1 < nbus ? sbm[b + 1].w : nt;
                int i = bm.w;
                double g = 0.0;
                if (i < tend) g = kk[2 * i++ + im];
                for (; i < tend; ++i) g += kk[2 * i + im];
                if (im) {   // <r_o, 2 v_o conj(Yd)> + (sum) / v_o
                    const double2 vw = sW[b], ro = sR[b], y = syd[b];
                    g = fma(g, vw.y, (vw.x + vw.x) * fma(ro.x, y.x, -ro.y * y.y));
                }
                spq[(im ? pqs : 0) + b + par] = g;
            }
        }
        if (a.aligned) {
            fence_proxy_async_smem();
            __syncthreads();
            if (tid == 0) {
                store_range_ll(a.gva, spq, sb + b0, sb + b0 + nbus);
                store_range_ll(a.gvm, spq + pqs, sb + b0, sb + b0 + nbus);
                bulk_commit();
                bulk_wait_read();
            }
        } else {
            __syncthreads();
            for (int b = tid; b < nbus; b += TB) {
                a.gva[sb + b0 + b] = spq[b + par];
                a.gvm[sb + b0 + b] = spq[pqs + b + par];
            }
        }
    }
    if (GRAD && !fused && a.gg)
        for (int l = l0 + TB; l < lr.y; l += TB) branch_grad(a, l, branch_const(a, l));
}

// ----------------------------------------------------------- launchers ----

static bool al16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

static BatchArgs batch_args(Batch *b)
{
    Grid *g = b->g;
    BatchArgs a = {};
    a.S = b->S;
    a.nb = g->nb;
    a.nl = g->nl;
    a.nnz = g->nnz;
    a.nwin = b->nwin;
    a.max_nbus = b->max_nbus;
    a.max_nt = b->max_nt;
    a.max_L = b->max_L;
    a.win_bus = b->win_bus;
    a.rorder = b->rorder;
    a.max_nph = b->max_nph;
    a.max_nbr = b->max_nbr;
    a.brl = b->brl;
    a.desc = b->desc;
    a.slotbus = b->slotbus;
    a.tloc = b->tloc;
    a.tp = g->tp;
    a.rp = g->rp;
    a.kd = g->kd;
    a.town = g->town;
    a.tmir = g->tmir;
    a.tpos = g->tpos;
    a.tnbr = g->tnbr;
    a.yd = g->bus_yd;
    a.tself = g->tself;
    a.tcoup = g->tcoup;
    a.tcfx = g->tcfx;
    a.tce = g->tce;
    a.trig = trig_table();
    a.sc = b->sc;
    a.joff = b->joff;
    a.U = b->U;
    a.V = b->V;
    a.bar = g->bar;
    a.err = g->err;
    a.r = b->r;
    a.lpart = b->lpart;
    a.pg = g->p_g;
    a.pb = g->p_b;
    a.pbsh = g->p_bsh;
    a.ptap = g->p_tap;
    a.pshift = g->p_shift;
    a.br_hk = g->br_hk;
    a.br_aux = g->br_aux;
    return a;
}

// Co-resident CTAs of `kernel` at tb threads and smem bytes (cached in resident).
template <typename K>
static cudaError_t coop_resident(K kernel, int &resident, int tb, size_t smem)
{
    cudaError_t e;
    if (resident == 0) {
        // set for every size: the kernels also hold a little static shared
        // memory, which counts against the default 48 KB
        if ((e = ensure_dyn_smem(reinterpret_cast<const void *>(kernel), smem))) return e;
        int per_sm = 0, dev = 0, nsm = 0;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, tb, smem))) return e;
        if ((e = cudaGetDevice(&dev)) || (e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)))
            return e;
        resident = per_sm * nsm;
        if (resident <= 0) return cudaErrorInvalidConfiguration;
    }
    return cudaSuccess;
}

// Cooperative launch of min(items, co-resident, cap) CTAs of tb threads (cap
// <= 0: none).
template <typename K>
static cudaError_t coop_launch(K kernel, int &resident, int tb, size_t smem, long long items, cudaStream_t s,
                               const BatchArgs &a, long long cap = 0)
{
    cudaError_t e = coop_resident(kernel, resident, tb, smem);
    if (e != cudaSuccess) return e;
    long long grid = std::min<long long>(items, resident);
    if (cap > 0) grid = std::min(grid, cap);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)std::max<long long>(1, grid));
    cfg.blockDim = dim3((unsigned)tb);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, a);
}

cudaError_t launch_ew_batched(Batch *b, bool jac, const double *vm, const double *va, double *P, double *Q,
                              double *J, cudaStream_t s)
{
    if (b->nwin == 0 || b->S == 0) return cudaSuccess;
    BatchArgs a = batch_args(b);
    a.vm = vm;
    a.va = va;
    a.P = P;
    a.Q = Q;
    a.J = J;
    a.aligned = (!J || al16(J)) && (!P || (al16(P) && al16(Q)));
    const EwSmem sp = ew_smem_plan(a.max_nbus, a.max_nt, jac ? a.max_L : 0, jac);
    const size_t smem = sp.total + kTrigSmem;
    const long long items = (long long)b->S * b->nwin;
    const long long cap = (long long)b->cfg.ctas_per_sm * b->nsm;
    if (jac) return coop_launch(k_ewb<true>, b->resident[1], b->tb, smem, items, s, a, cap);
    return coop_launch(k_ewb<false>, b->resident[0], b->tb, smem, items, s, a, cap);
}

// The adjoint (grad) or the loss alone: one item per CTA (k_adj1) when every
// (scenario, window) item fits on the GPU at once, else the throughput form.
template <bool GRAD>
static cudaError_t launch_adj(Batch *b, BatchArgs &a, cudaStream_t s)
{
    Grid *g = b->g;
    const long long items = (long long)b->S * b->nwin;
    const int r1 = GRAD ? 3 : 5, rn = GRAD ? 2 : 4;   // resident-CTA caches of the four kernels
    const long long branch_ctas1 = GRAD ? (g->nl + kAdj1Threads - 1) / kAdj1Threads : 0;
    const long long branch_ctas = GRAD ? (g->nl + b->tb - 1) / b->tb : 0;
    if (b->ghost && b->cfg.adjoint_form == 0) {
        // the form is chosen by the gradient kernel's residency for both, so that
        // the loss alone and the adjoint sum the same terms in the same order
        const size_t smem = adj1_smem_plan(a.max_nbus, a.max_nt, a.max_nph).total;
        cudaError_t e = coop_resident(k_adj1<true>, b->resident[3], kAdj1Threads, smem);
        if (e == cudaSuccess) e = coop_resident(k_adj1<GRAD>, b->resident[r1], kAdj1Threads, smem);
        if (e != cudaSuccess) return e;
        if (items <= b->resident[3])
            return coop_launch(k_adj1<GRAD>, b->resident[r1], kAdj1Threads, smem,
                               std::max<long long>(items, branch_ctas1), s, a);
    }
    const size_t smem = ew_smem_plan(a.max_nbus, a.max_nt, 0, false).total + kTrigSmem;
    return coop_launch(k_adj<GRAD>, b->resident[rn], b->tb, smem, std::max<long long>(items, branch_ctas), s, a,
                       (long long)b->cfg.ctas_per_sm * b->nsm);
}

static BatchArgs loss_args(Batch *b, const double *vm, const double *va, const double *Ps, const double *Qs,
                           const double *wP, const double *wQ, double *L, double *Ltot)
{
    BatchArgs a = batch_args(b);
    a.vm = vm;
    a.va = va;
    a.Ps = Ps;
    a.Qs = Qs;
    a.wP = wP;
    a.wQ = wQ;
    a.L = L ? L : b->lscen;   // the total needs every L_s somewhere
    a.Ltot = Ltot;
    a.lcnt = b->g->bar + kLossCountWord;
    return a;
}

cudaError_t launch_adjoint(Batch *b, const double *vm, const double *va, const double *Ps, const double *Qs,
                           const double *wP, const double *wQ, const double *Lbar, double *L, double *Ltot,
                           double *gvm, double *gva, double *gg, double *gb, double *gbsh, double *gtap,
                           cudaStream_t s)
{
    if (b->nwin == 0 || b->S == 0) return cudaSuccess;
    BatchArgs a = loss_args(b, vm, va, Ps, Qs, wP, wQ, L, Ltot);
    a.Lbar = Lbar;
    a.gvm = gvm;
    a.gva = gva;
    a.gg = gg;
    a.gb = gb;
    a.gbsh = gbsh;
    a.gtap = gtap;
    a.aligned = al16(gvm) && al16(gva);
    return launch_adj<true>(b, a, s);
}

cudaError_t launch_loss(Batch *b, const double *vm, const double *va, const double *Ps, const double *Qs,
                        const double *wP, const double *wQ, double *L, double *Ltot, cudaStream_t s)
{
    if (b->nwin == 0 || b->S == 0) return cudaSuccess;
    BatchArgs a = loss_args(b, vm, va, Ps, Qs, wP, wQ, L, Ltot);
    return launch_adj<false>(b, a, s);
}

}  // namespace pf
