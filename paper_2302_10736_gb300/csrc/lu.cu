// lu.cu - sparse LU solve of the reduced Newton system J_r dx = F on the GPU
// (the paper hands the Jacobian to a sparse direct solver, KLU, and does not
// study the solve; this is this library's own).
//
// Analysis (host, once per set of bus types):
//   * J_r is structurally symmetric when equation P_i is paired with unknown
//     theta_i and Q_i with v_i, so its pattern is that of a graph on the
//     buses; the buses are ordered by minimum degree (each elimination joins
//     the eliminated bus's neighbours into a clique; ties to the lowest bus),
//     which keeps the factor close to the matrix on power grids (about 1.5
//     times its entries on the synthetic grids), and a bus's unknowns stay
//     adjacent (theta, then v).
//   * Symbolic factorization of the permuted pattern: the elimination tree and
//     the pattern of L by row subtrees; U has the transposed pattern, so one
//     index structure (CSC of L) serves both factors: Lx[p] = L(Li[p], j) and
//     Ux[p] = U(j, Li[p]) for p in Lp[j] .. Lp[j+1].
//   * The columns grouped by height in the elimination tree: a column depends
//     only on its descendants, which are all lower.
//
// Numeric phase (GPU), left-looking Crout factorization without pivoting in
// gather form: the analysis lists, for every factor slot (i, j), the pairs of
// slots (L(i, k), U(k, j)) - and for the mirrored U(j, i) the pairs
// (L(j, k), U(k, i)) - over the k below j that update it, ascending, so every
// slot is one independent sum:
//   d   = A(j, j) - sum_k L(j, k) U(k, j)          U(j, j) = d
//   y_j = F_j    - sum_k L(j, k) y_k               (forward solve, fused)
//   L(i, j) = (A(i, j) - sum_k L(i, k) U(k, j)) / d,  U(j, i) = A(j, i) - sum_k L(j, k) U(k, i)
// then the backward solve x_j = (y_j - sum_i U(j, i) x_i) / U(j, j) from the
// root down.
//
// The dynamic schedule (k_lu_solve, a cooperative launch).  No barrier
// separates the levels: a column depends only on its descendants in the
// elimination tree, so every work item waits for its column's children to be
// finished (per-column counters, bounded waits) and the work runs as soon as
// its inputs exist, along the tree's critical path rather than level by level.
// Work items are in level order and the warps take them in that order from a
// shared counter, so the lowest unfinished item has a warp and its inputs, and
// can always run (all CTAs are resident: cooperative launch).  Wide levels
// give a warp to a column (a lane per slot); on the upper levels (those with
// no more slots than the launch has warps) every slot of a column gets a warp
// of its own (its lanes splitting the slot's sum; each warp forms its
// column's pivot itself, the same way); the backward solve gives a warp to a
// column, which waits for its own factorization and then for its parent.
// What an item needs that no other item writes - its index lists and its own
// slots' values of A and F - is loaded before its wait, and after the wait all
// its loads of other columns' factor values are in flight at once (four terms
// per lane), so a level of the tree costs one round trip to L2 for the values,
// one for the release of the results and one for the next item's acquire.
// Values written by other CTAs are read with L1-bypassing loads after an
// acquire load of the counter that announced them.
//
// The tail (k_lu_tail, one thread-block cluster).  At the top of the tree the
// levels hold one or two columns each, and the schedule above would pay a
// chain of round trips per column.  The longest run of final columns T0 .. n-1
// on such levels (closed under the tree's ancestors) is factored as a dense
// block in the cluster's shared memory; the dynamic launch computes only its
// entries' terms over the columns outside it (parallel items, after the tail's
// frontier is finished), and a second dynamic launch solves backward below it.
// Without a tail (fewer than kLuTailMin such columns) one launch does it all.
//
// Every sum has a fixed order (sequential, or lane-strided partial sums joined
// by a fixed shuffle tree): the results are bitwise repeatable.  A zero or
// non-finite pivot sets the grid's error word (no trap); a wait that runs out
// (2 s) sets it to a time-out and ends the warp.
#include <algorithm>
#include <set>
#include <vector>

#include <cooperative_groups.h>

#include "fastmath.cuh"
#include "pf_internal.h"
#include "ptx.cuh"

namespace pf {

namespace {

constexpr uint64_t kLuBarrierNs = 2000000000ull;   // bounded grid-barrier wait (2 s)
constexpr int kLuThreads = 384;
// the tail: the top of the elimination tree factored as a dense block by one
// thread-block cluster (shared memory spread over its CTAs)
constexpr int kLuTailCtas = 8;
constexpr int kLuTailThreads = 512;
constexpr int kLuTailMax = 384;   // columns: 48 rows of 384 doubles per CTA
constexpr int kLuTailMin = 16;    // a shorter top chain stays in the dynamic schedule
constexpr int kLuTailWidth = 2;   // the tail holds columns of levels at most this wide

struct LuArgs {
    int n, nnzA, nfitems, nbcols;
    int T0, LpT0;   // the tail's first column and first factor slot (n, nnz(L): no tail)
    int fr0, fr1;   // the tail's frontier in cidx: the columns outside it whose parent is in it
    int mode;       // 0 the whole solve; 1 zero, scatter, factorization (the tail's outside terms only); 2 the backward solve outside the tail
    const int *Lp, *Li, *Rp, *Rk, *Rq, *perm, *amap, *gptr;
    const int *need, *cptr, *cidx, *parent, *bcols;
    const int2 *gsrc;     // per update term of a slot: {L(i, k) slot, U(k, j) slot}
    const int2 *fitems;   // {column, -2 (whole column) or slot or -1 (pivot only)}, level order
    const double *A, *F;
    double *Lx, *Ux, *D, *y, *dx;
    double *piv;          // [n] the pivots U(j, j) (D keeps A(j, j): every item of a column reads it)
    int *done;            // [2n + 2]: finished items of column j at j, x_j written at n + j, the item counters
    unsigned int *bar;
    int *err;
};

__device__ __forceinline__ int ld_acquire(const int *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long lu_gtimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// wait until *p >= target, at most kLuBarrierNs; false (and the grid's error
// word set to a time-out) if it never gets there
__device__ __forceinline__ bool lu_wait(const LuArgs &a, const int *p, int target)
{
    if (ld_acquire(p) >= target) return true;
    const unsigned long long t0 = lu_gtimer();
    for (;;) {
        __nanosleep(20);
        if (ld_acquire(p) >= target) return true;
        if (lu_gtimer() - t0 > kLuBarrierNs) {
            atomicExch(a.err, DEV_TIMEOUT);
            return false;
        }
    }
}

// every child of column j in the elimination tree finished (the lanes wait for
// different children); false on a time-out (all lanes agree)
__device__ __forceinline__ bool lu_wait_children(const LuArgs &a, int j, int lane)
{
    bool ok = true;
    // a column of the tail reads the outside columns of its whole subtree: it
    // waits for the tail's frontier
    const int c0 = j >= a.T0 ? a.fr0 : a.cptr[j], c1 = j >= a.T0 ? a.fr1 : a.cptr[j + 1];
    for (int t = c0 + lane; t < c1; t += 32) {
        const int c = a.cidx[t];
        ok = ok && lu_wait(a, a.done + c, a.need[c]);
    }
    ok = __all_sync(0xffffffffu, ok);
    __syncwarp();   // orders the waiting lanes' acquires before every lane's reads
    return ok;
}

// the warp's writes visible, then one more finished item of column j
__device__ __forceinline__ void lu_finish(const LuArgs &a, int *cnt, int lane)
{
    __threadfence();
    __syncwarp();
    if (lane == 0) atomicAdd(cnt, 1);
}

__device__ __forceinline__ double ldcg(const double *p) { return __ldcg(p); }

__device__ __forceinline__ double warp_sum_d(double x)
{
    for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
    return x;
}

__device__ __forceinline__ void pivot_check(const LuArgs &a, double d)
{
    if (!(fabs(d) > 0.0) || !isfinite(d)) atomicExch(a.err, DEV_SINGULAR);
}

// The static part of a work item - index lists fixed by the analysis, and the
// values of A and F in the item's own slots, which no other item writes - is
// loaded before the item's wait, so that after it only the factor values of
// its descendants remain to be read (one round trip instead of three).

// row j's (slot, column) pairs, the first 128 (four per lane, lane-strided)
struct LuRow {
    int r, r1;   // the next entry after the loaded ones, the row's end
    int q[4], k[4];
};

__device__ __forceinline__ void lu_row_load(const LuArgs &a, int j, int lane, LuRow &w)
{
    const int r0 = a.Rp[j] + lane;
    w.r1 = a.Rp[j + 1];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int r = r0 + 32 * u;
        w.k[u] = r < w.r1 ? a.Rk[r] : 0;
        w.q[u] = r < w.r1 && w.k[u] < a.T0 ? a.Rq[r] : -1;   // k in the tail: the dense phase's term
    }
    w.r = r0 + 128;
}

// a slot's update pairs {L(i, k) slot, U(k, j) slot}, the first four of the
// lane's share: lane-strided (`stride` 32, a warp per slot) or consecutive
// (`stride` 1, a lane per slot)
struct LuSlot {
    int g, g1;
    int2 s[4];
};

__device__ __forceinline__ void lu_slot_load(const LuArgs &a, int p, int g0, int stride, LuSlot &w)
{
    w.g1 = a.gptr[p + 1];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int g = g0 + stride * u;
        w.s[u] = g < w.g1 ? a.gsrc[g] : make_int2(-1, -1);
        if (w.s[u].y >= a.LpT0) w.s[u] = make_int2(-1, -1);   // k in the tail: the dense phase's term
    }
    w.g = g0 + 4 * stride;
}

// the values of the loaded pairs (after the wait)
struct LuRowVal {
    double l[4], uu[4], yk[4];
};
struct LuSlotVal {
    double lx[4], uy[4], ly[4], ux[4];
};

// (a term the lane does not have reads as 0 x 0, which leaves a sum unchanged
// but for the sign of a zero; the indices are not needed after the loads)
__device__ __forceinline__ void lu_row_fetch(const LuArgs &a, const LuRow &w, bool fwd, LuRowVal &v)
{
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const bool h = w.q[u] >= 0;
        v.l[u] = h ? ldcg(a.Lx + w.q[u]) : 0.0;
        v.uu[u] = h ? ldcg(a.Ux + w.q[u]) : 0.0;
        v.yk[u] = h && fwd ? ldcg(a.y + w.k[u]) : 0.0;
    }
}

__device__ __forceinline__ void lu_slot_fetch(const LuArgs &a, const LuSlot &w, LuSlotVal &v)
{
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const bool h = w.s[u].x >= 0;
        v.lx[u] = h ? ldcg(a.Lx + w.s[u].x) : 0.0;
        v.uy[u] = h ? ldcg(a.Ux + w.s[u].y) : 0.0;
        v.ly[u] = h ? ldcg(a.Lx + w.s[u].y) : 0.0;
        v.ux[u] = h ? ldcg(a.Ux + w.s[u].x) : 0.0;
    }
}

// the lane's part of sum_k L(j, k) U(k, j) and sum_k L(j, k) y_k: the fetched
// four (first), then the rest of its share of row j, four in flight (rest);
// lane-strided, so every lane adds its terms in ascending order
__device__ __forceinline__ double2 lu_row_first(const LuRowVal &v)
{
    double dd = 0.0, yy = 0.0;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        dd = fma(v.l[u], v.uu[u], dd);
        yy = fma(v.l[u], v.yk[u], yy);
    }
    return make_double2(dd, yy);
}

__device__ __forceinline__ double2 lu_row_rest(const LuArgs &a, const LuRow &w, double2 t)
{
    double dd = t.x, yy = t.y;
    #pragma unroll 1
    for (int r = w.r; r < w.r1; r += 128) {
        int q[4], k[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            k[u] = r + 32 * u < w.r1 ? a.Rk[r + 32 * u] : 0;
            q[u] = r + 32 * u < w.r1 && k[u] < a.T0 ? a.Rq[r + 32 * u] : -1;
        }
        double l[4], uu[4], yk[4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (q[u] >= 0) {
                l[u] = ldcg(a.Lx + q[u]);
                uu[u] = ldcg(a.Ux + q[u]);
                yk[u] = ldcg(a.y + k[u]);
            }
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (q[u] >= 0) {
                dd = fma(l[u], uu[u], dd);
                yy = fma(l[u], yk[u], yy);
            }
    }
    return make_double2(dd, yy);
}

// sl - sum L(i, k) U(k, j) and su - sum L(j, k) U(k, i) over the lane's share
// of a slot's pairs: the fetched four (first), then the rest (`stride` as
// loaded), four in flight, in ascending order (rest)
__device__ __forceinline__ double2 lu_slot_first(const LuSlotVal &v, double sl, double su)
{
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        sl = fma(-v.lx[u], v.uy[u], sl);
        su = fma(-v.ly[u], v.ux[u], su);
    }
    return make_double2(sl, su);
}

__device__ __forceinline__ double2 lu_slot_rest(const LuArgs &a, const LuSlot &w, int stride, double2 t)
{
    double sl = t.x, su = t.y;
    #pragma unroll 1
    for (int g = w.g; g < w.g1; g += 4 * stride) {
        int2 s4[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            s4[u] = g + stride * u < w.g1 ? a.gsrc[g + stride * u] : make_int2(-1, -1);
            if (s4[u].y >= a.LpT0) s4[u] = make_int2(-1, -1);
        }
        double lx[4], uy[4], ly[4], ux[4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (s4[u].x >= 0) {
                lx[u] = ldcg(a.Lx + s4[u].x);
                uy[u] = ldcg(a.Ux + s4[u].y);
                ly[u] = ldcg(a.Lx + s4[u].y);
                ux[u] = ldcg(a.Ux + s4[u].x);
            }
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (s4[u].x >= 0) {
                sl = fma(-lx[u], uy[u], sl);
                su = fma(-ly[u], ux[u], su);
            }
    }
    return make_double2(sl, su);
}

// A factorization item's static part: its row (the pivot and forward terms),
// and either the lane's first slot of column j (a warp per column: p0 = -2)
// or the slot's first pairs (a warp per slot p0 = p >= 0; -1: no slot), with
// A(j, j), F_j's place in y and the slot's values of A
struct LuItem {
    LuRow row;
    LuSlot slot;
    int j, p, pfirst, pend;   // column; the lane's (column warp) or the item's slot (-1: none); column j's slots
    bool colwarp;
    double d0, y0, l0, u0;    // A(j, j), y_j before the update, the slot's A values (the lane sums' start)
};

__device__ __forceinline__ void lu_item_load(const LuArgs &a, int j, int p0, int lane, LuItem &it)
{
    it.j = j;
    it.colwarp = p0 == -2;
    lu_row_load(a, j, lane, it.row);
    it.pfirst = a.Lp[j];
    it.pend = a.Lp[j + 1];
    it.d0 = ldcg(a.D + j);
    it.y0 = ldcg(a.y + j);
    it.p = it.colwarp ? (it.pfirst + lane < it.pend ? it.pfirst + lane : -1) : p0;
    it.l0 = it.u0 = 0.0;
    it.slot.g = it.slot.g1 = 0;
#pragma unroll
    for (int u = 0; u < 4; ++u) it.slot.s[u] = make_int2(-1, -1);
    if (it.p >= 0) {
        const int g0 = a.gptr[it.p];
        lu_slot_load(a, it.p, it.colwarp ? g0 : g0 + lane, it.colwarp ? 1 : 32, it.slot);
        it.l0 = ldcg(a.Lx + it.p);
        it.u0 = ldcg(a.Ux + it.p);
    }
}

// One factorization item by one warp, after its wait.  A whole column (wide
// levels, `it.colwarp`): its pivot, then a lane per slot, each slot's update
// terms in order, four in flight.  One slot of a narrow level's column (p < 0:
// the column has no slot below the diagonal): the lanes split the slot's
// terms; every item of a column forms its pivot the same way, and the
// column's first item also writes the pivot and y_j.  A column of the tail
// (j >= T0) takes only the terms of columns outside it and keeps its
// numerators, pivot and y_j unfinished for the dense phase.
__device__ __forceinline__ void lu_factor(const LuArgs &a, const LuItem &it, int lane)
{
    const bool tail = it.j >= a.T0;
    // y_j is formed by a column warp and by a column's first item only
    const bool fwd = it.colwarp || it.p < 0 || it.p == it.pfirst;
    LuRowVal rv;
    LuSlotVal sv;
    lu_row_fetch(a, it.row, fwd, rv);
    lu_slot_fetch(a, it.slot, sv);
    double2 t = lu_row_first(rv);
    // a lane's own slot (column warp) starts from A's values, the lane sums of
    // a warp's slot from 0
    double2 s = lu_slot_first(sv, it.colwarp ? it.l0 : 0.0, it.colwarp ? it.u0 : 0.0);
    t = lu_row_rest(a, it.row, t);
    s = lu_slot_rest(a, it.slot, it.colwarp ? 1 : 32, s);
    const double d = it.d0 - warp_sum_d(t.x), yj = it.y0 - warp_sum_d(t.y);
    const double inv = fast_rcp(d);
    if (it.colwarp) {
        if (it.p >= 0) {
            a.Lx[it.p] = s.x * inv;
            a.Ux[it.p] = s.y;
            // slots beyond the warp's first 32
#pragma unroll 1
            for (int p = it.p + 32; p < it.pend; p += 32) {
                LuSlot w;
                w.g = a.gptr[p];
                w.g1 = a.gptr[p + 1];
                const double2 s2 = lu_slot_rest(a, w, 1, make_double2(ldcg(a.Lx + p), ldcg(a.Ux + p)));
                a.Lx[p] = s2.x * inv;
                a.Ux[p] = s2.y;
            }
        }
    } else if (it.p >= 0) {
        // the lane sums were formed as 0 - terms: their warp sum is minus the
        // slot's sum
        const double sx = warp_sum_d(s.x), sy = warp_sum_d(s.y);
        if (lane == 0) {
            a.Lx[it.p] = tail ? it.l0 + sx : (it.l0 + sx) * inv;
            a.Ux[it.p] = it.u0 + sy;
        }
    }
    if (lane == 0 && fwd) {
        if (!tail) pivot_check(a, d);
        a.piv[it.j] = d;
        a.y[it.j] = yj;
    }
}

// x_j of the backward solve, in place of y_j (one warp): the column's rows are
// loaded before any wait, its U values, y_j and pivot once its own
// factorization is finished, the x of its rows (its ancestors) once its
// parent's x is written; false on a time-out (all lanes agree)
__device__ __forceinline__ bool lu_back(const LuArgs &a, int j, int lane)
{
    const int p0 = a.Lp[j] + lane, p1 = a.Lp[j + 1], pj = a.parent[j], need = a.need[j], pm = a.perm[j];
    int li[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) li[u] = p0 + 32 * u < p1 ? a.Li[p0 + 32 * u] : -1;
    if (!__all_sync(0xffffffffu, lu_wait(a, a.done + j, need))) return false;
    __syncwarp();
    double ux[4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
        if (li[u] >= 0) ux[u] = ldcg(a.Ux + p0 + 32 * u);
    const double yj = ldcg(a.y + j), pv = ldcg(a.piv + j);
    if (pj >= 0) {
        if (!__all_sync(0xffffffffu, lu_wait(a, a.done + a.n + pj, 1))) return false;
        __syncwarp();
    }
    double s = 0.0;
#pragma unroll
    for (int u = 0; u < 4; ++u)
        if (li[u] >= 0) s = fma(ux[u], ldcg(a.y + li[u]), s);
    #pragma unroll 1
    for (int p = p0 + 128; p < p1; p += 32) s = fma(ldcg(a.Ux + p), ldcg(a.y + a.Li[p]), s);
    s = warp_sum_d(s);
    if (lane == 0) {
        const double x = (yj - s) * fast_rcp(pv);
        a.y[j] = x;
        a.dx[pm] = x;
    }
    return true;
}

__global__ void __launch_bounds__(kLuThreads) k_lu_solve(LuArgs a)
{
    const GridBar gbar = a.mode != 2 ? grid_barrier_begin(a.bar) : GridBar{nullptr, 0u};
    const int lane = threadIdx.x & 31;
    const long long gtid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long gthreads = (long long)gridDim.x * blockDim.x;
    const int nnzL = a.Lp[a.n];
    unsigned int bk = 0;
    if (a.mode != 2) {
        // ---- the factor storage and the counters zeroed, then A and the
        // right-hand side scattered in ----
        for (long long t = gtid; t < nnzL; t += gthreads) {
            a.Lx[t] = 0.0;
            a.Ux[t] = 0.0;
        }
        for (long long t = gtid; t < 2LL * a.n + 2; t += gthreads) a.done[t] = 0;   // and the item counters
        if (!grid_barrier(gbar, a.bar, gridDim.x, bk++, a.err, DEV_TIMEOUT, kLuBarrierNs)) return;
        for (long long e = gtid; e < a.nnzA; e += gthreads) {
            const int code = a.amap[e], slot = code >> 2;
            const double v = a.A[e];
            if ((code & 3) == 0)
                a.Lx[slot] = v;
            else if ((code & 3) == 1)
                a.Ux[slot] = v;
            else
                a.D[slot] = v;
        }
        for (long long j = gtid; j < a.n; j += gthreads) a.y[j] = a.F[a.perm[j]];
        if (!grid_barrier(gbar, a.bar, gridDim.x, bk++, a.err, DEV_TIMEOUT, kLuBarrierNs)) return;
    }
    // ---- every warp takes the next item (factorization and forward solve in
    // level order, then the backward solve from the root down) from a shared
    // counter, waits for what the item depends on, and runs it ----
    int *next = a.done + 2LL * a.n + (a.mode == 2 ? 1 : 0);
    const int nf = a.mode == 2 ? 0 : a.nfitems;
    const int nall = nf + (a.mode == 1 ? 0 : a.nbcols);
    for (;;) {
        int t = 0;
        if (lane == 0) t = atomicAdd(next, 1);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= nall) break;
        if (t < nf) {   // once the column's children are finished
            const int2 fi = a.fitems[t];
            LuItem it;
            lu_item_load(a, fi.x, fi.y, lane, it);
            if (!lu_wait_children(a, fi.x, lane)) return;
            lu_factor(a, it, lane);
            lu_finish(a, a.done + fi.x, lane);
        } else {   // x_j once its own factorization is finished and its parent's x is written
            const int j = a.bcols[t - nf];
            if (!lu_back(a, j, lane)) return;
            lu_finish(a, a.done + a.n + j, lane);
        }
    }
}

// The tail (columns T0 .. n-1, the top of the elimination tree, where the
// dynamic schedule would pay a chain of L2 round trips per column) as a dense
// block of m = n - T0 rows and columns, by one cluster of kLuTailCtas CTAs:
// row i of the block lives in the shared memory of CTA i mod C (row-cyclic,
// so every step's rows are spread over all CTAs), and the CTAs read the
// current pivot row, y_k and x_k from each other's shared memory.  On entry
// the tail's slots hold A's values less the terms of the columns outside the
// tail (L numerators, U values, the pivots' and y's partial sums); the kernel
// finishes them right-looking in the same order of terms as a column of the
// dynamic schedule (k ascending, one fused multiply-add per term), solving
// L y = F on the way, then solves U x = y backward, writes x_j into y_j and
// dx, and marks the tail's x written for the backward solve below it.  One
// cluster barrier per step (a warp per row in the factorization, a thread per
// row in the backward solve, so that no other barrier is needed there).
// Cluster barriers are hardware barriers every CTA passes the same number of
// times.
__global__ void __cluster_dims__(kLuTailCtas, 1, 1) __launch_bounds__(kLuTailThreads, 1) k_lu_tail(LuArgs a)
{
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    extern __shared__ __align__(16) double tsm[];
    constexpr int C = kLuTailCtas;
    const int rank = (int)cl.block_rank();
    const int T0 = a.T0, m = a.n - T0, R = (m + C - 1) / C;
    const int tid = threadIdx.x, TB = blockDim.x, lane = tid & 31, wid = tid >> 5, nw = TB >> 5;
    double *S = tsm;                        // [R][m]: block rows rank, rank + C, rank + 2C, ...
    double *yv = S + (size_t)R * m;         // [R] y, then the right-hand side of the backward solve
    double *xl = yv + R;                    // [R] x
    double *prow = xl + R;                  // [m + 1] the current pivot row (columns k .. m-1) and y_k
    const int nown = rank < m ? (m - 1 - rank) / C + 1 : 0;   // rows of this CTA
    // ---- the block: column jj's slots give L(ii, jj) to row ii's CTA and
    // U(jj, ii) to row jj's ----
    for (int t = tid; t < R * m; t += TB) S[t] = 0.0;
    __syncthreads();
    for (int jj = wid; jj < m; jj += nw) {
        const int j = T0 + jj;
        for (int p = a.Lp[j] + lane; p < a.Lp[j + 1]; p += 32) {
            const int ii = a.Li[p] - T0;
            if (ii % C == rank) S[(size_t)(ii / C) * m + jj] = __ldcg(a.Lx + p);
            if (jj % C == rank) S[(size_t)(jj / C) * m + ii] = __ldcg(a.Ux + p);
        }
        if (lane == 0 && jj % C == rank) {
            S[(size_t)(jj / C) * m + jj] = __ldcg(a.piv + j);
            yv[jj / C] = __ldcg(a.y + j);
        }
    }
    cl.sync();
    // ---- factorization and forward solve, one pivot per step: the pivot row
    // copied in, then a warp per row below it ----
    for (int k = 0; k < m; ++k) {
        const int own = k % C, kr = k / C;
        const double *Sk = cl.map_shared_rank(S, own) + (size_t)kr * m;
        for (int c = k + tid; c < m; c += TB) prow[c] = Sk[c];
        if (tid == TB - 1) prow[m] = *cl.map_shared_rank(yv + kr, own);
        __syncthreads();
        const double d = prow[k], inv = fast_rcp(d), yk = prow[m];
        if (rank == own && tid == 0) pivot_check(a, d);
        for (int r = (k + C - rank) / C + wid; r < nown; r += nw) {   // this CTA's rows below k
            double *Sr = S + (size_t)r * m;
            const double l = Sr[k] * inv;
            for (int c = k + 1 + lane; c < m; c += 32) Sr[c] = fma(-l, prow[c], Sr[c]);
            __syncwarp();
            if (lane == 0) {
                Sr[k] = l;
                yv[r] = fma(-l, yk, yv[r]);
            }
        }
        cl.sync();
    }
    // ---- backward solve: thread r keeps row r's right-hand side; x_k by the
    // thread of row k, then every row above k takes its term out ----
    for (int k = m - 1; k >= 0; --k) {
        const int own = k % C, kr = k / C;
        if (rank == own && tid == kr) xl[kr] = yv[kr] * fast_rcp(S[(size_t)kr * m + k]);
        cl.sync();
        if (tid < nown && tid * C + rank < k)
            yv[tid] = fma(-S[(size_t)tid * m + k], *cl.map_shared_rank(xl + kr, own), yv[tid]);
    }
    // ---- x out, and the tail's x marked written ----
    for (int r = tid; r < nown; r += TB) {
        const int j = T0 + r * C + rank;
        a.y[j] = xl[r];
        a.dx[a.perm[j]] = xl[r];
        a.done[a.n + j] = 1;
    }
    cl.sync();   // no CTA leaves while another may still read its shared memory
}

// shared memory of k_lu_tail for a tail of m columns
size_t lu_tail_smem(int m)
{
    const size_t R = (size_t)(m + kLuTailCtas - 1) / kLuTailCtas;
    return sizeof(double) * (R * (size_t)m + 2 * R + (size_t)m + 1);
}

// ------------------------------------------------------------ analysis ----

// Minimum-degree order of an undirected graph (explicit elimination: the
// neighbours of each eliminated node become a clique; ties to the lowest node).
std::vector<int> min_degree_order(std::vector<std::vector<int>> adj)
{
    const int n = (int)adj.size();
    std::set<std::pair<int, int>> pq;
    for (int u = 0; u < n; ++u) pq.insert({(int)adj[u].size(), u});
    std::vector<char> gone(n, 0);
    std::vector<int> order;
    order.reserve(n);
    std::vector<int> merged;
    while (!pq.empty()) {
        const int u = pq.begin()->second;
        pq.erase(pq.begin());
        gone[u] = 1;
        order.push_back(u);
        const std::vector<int> nb = adj[u];   // sorted, live nodes only
        for (int v : nb) {
            pq.erase({(int)adj[v].size(), v});
            merged.clear();
            std::set_union(adj[v].begin(), adj[v].end(), nb.begin(), nb.end(), std::back_inserter(merged));
            adj[v].clear();
            for (int x : merged)
                if (x != v && x != u) adj[v].push_back(x);
            pq.insert({(int)adj[v].size(), v});
        }
        adj[u].clear();
        adj[u].shrink_to_fit();
    }
    return order;
}

}  // namespace

pf_status host_lu(int nb, int n, int npvpq, const std::vector<int> &colptr, const std::vector<int> &rowidx,
                  const std::vector<int> &fmap, int slot_warps, HostLu &L)
{
    L = HostLu{};
    L.n = n;
    // bus graph of the unknowns' buses (every unknown's bus has a theta unknown)
    std::vector<int> node(nb, -1), bus_of;
    for (int k = 0; k < npvpq; ++k) {
        node[fmap[k]] = (int)bus_of.size();
        bus_of.push_back(fmap[k]);
    }
    const int B = (int)bus_of.size();
    std::vector<std::vector<int>> adj(B);
    for (int c = 0; c < n; ++c)
        for (int p = colptr[c]; p < colptr[c + 1]; ++p) {
            const int u = node[fmap[rowidx[p]]], v = node[fmap[c]];
            if (u < 0 || v < 0) return set_error(PF_EINVAL, "jac_reduced_solve: an unknown without a bus angle");
            if (u != v) {
                adj[u].push_back(v);
                adj[v].push_back(u);
            }
        }
    for (auto &a : adj) {
        std::sort(a.begin(), a.end());
        a.erase(std::unique(a.begin(), a.end()), a.end());
    }
    const std::vector<int> border = min_degree_order(adj);
    // unknowns in elimination order: each bus's theta, then its v
    std::vector<int> vidx(nb, -1);
    for (int k = npvpq; k < n; ++k) vidx[fmap[k]] = k;
    L.perm.reserve(n);
    std::vector<int> tidx(nb, -1);
    for (int k = 0; k < npvpq; ++k) tidx[fmap[k]] = k;
    for (int u : border) {
        const int b = bus_of[u];
        L.perm.push_back(tidx[b]);
        if (vidx[b] >= 0) L.perm.push_back(vidx[b]);
    }
    if ((int)L.perm.size() != n) return set_error(PF_EINVAL, "jac_reduced_solve: unknowns do not match buses");
    std::vector<int> iperm(n);
    for (int i = 0; i < n; ++i) iperm[L.perm[i]] = i;
    // lower pattern of the permuted (symmetrised) matrix, row by row
    std::vector<std::vector<int>> low(n);
    for (int c = 0; c < n; ++c)
        for (int p = colptr[c]; p < colptr[c + 1]; ++p) {
            const int i = iperm[rowidx[p]], j = iperm[c];
            if (i > j) low[i].push_back(j);
            if (j > i) low[j].push_back(i);
        }
    for (auto &r : low) {
        std::sort(r.begin(), r.end());
        r.erase(std::unique(r.begin(), r.end()), r.end());
    }
    // elimination tree and the rows of L by row subtrees
    std::vector<int> parent(n, -1), flag(n, -1), cnt(n, 0);
    std::vector<std::vector<int>> lrow(n);
    for (int i = 0; i < n; ++i) {
        flag[i] = i;
        for (int k : low[i]) {
            while (k != -1 && flag[k] != i) {
                if (parent[k] == -1) parent[k] = i;
                lrow[i].push_back(k);
                cnt[k]++;
                flag[k] = i;
                k = parent[k];
            }
        }
        std::sort(lrow[i].begin(), lrow[i].end());
    }
    L.Lp.assign(n + 1, 0);
    for (int j = 0; j < n; ++j) L.Lp[j + 1] = L.Lp[j] + cnt[j];
    const long long nnzL = L.Lp[n];
    if (nnzL >= (1LL << 29)) return set_error(PF_EUNSUPPORTED, "jac_reduced_solve: factor too large");
    L.Li.assign(nnzL, 0);
    L.Rp.assign(n + 1, 0);
    L.Rk.reserve(nnzL);
    L.Rq.reserve(nnzL);
    std::vector<int> fill(L.Lp.begin(), L.Lp.end() - 1);
    for (int i = 0; i < n; ++i) {   // rows ascending: every column's rows come out ascending
        for (int k : lrow[i]) {
            L.Rk.push_back(k);
            L.Rq.push_back(fill[k]);
            L.Li[fill[k]++] = i;
        }
        L.Rp[i + 1] = (int)L.Rk.size();
        std::vector<int>().swap(lrow[i]);
    }
    // the update terms of every slot p = (i, j) of column j: for each k of row j
    // (ascending), the pairs {slot of L(i, k), slot of L(j, k)} over the rows i of
    // column k below j (all of them are in column j's pattern)
    auto slot_of = [&](int col, int row) {
        const auto b = L.Li.begin() + L.Lp[col], e = L.Li.begin() + L.Lp[col + 1];
        return (int)(std::lower_bound(b, e, row) - L.Li.begin());
    };
    L.gptr.assign(nnzL + 1, 0);
    for (int j = 0; j < n; ++j)
        for (int r = L.Rp[j]; r < L.Rp[j + 1]; ++r) {
            const int k = L.Rk[r], q = L.Rq[r];
            for (int pp = q + 1; pp < L.Lp[k + 1]; ++pp) L.gptr[slot_of(j, L.Li[pp]) + 1]++;
        }
    for (long long p = 0; p < nnzL; ++p) L.gptr[p + 1] += L.gptr[p];
    if (L.gptr[nnzL] >= (1LL << 30)) return set_error(PF_EUNSUPPORTED, "jac_reduced_solve: factorization too large");
    L.gsrc.assign(L.gptr[nnzL], make_int2(0, 0));
    {
        std::vector<int> gf(L.gptr.begin(), L.gptr.end() - 1);
        for (int j = 0; j < n; ++j)
            for (int r = L.Rp[j]; r < L.Rp[j + 1]; ++r) {
                const int k = L.Rk[r], q = L.Rq[r];
                for (int pp = q + 1; pp < L.Lp[k + 1]; ++pp) L.gsrc[gf[slot_of(j, L.Li[pp])]++] = make_int2(pp, q);
            }
    }
    // levels by height in the tree
    std::vector<int> height(n, 0);
    for (int j = 0; j < n; ++j)
        if (parent[j] >= 0) height[parent[j]] = std::max(height[parent[j]], height[j] + 1);
    L.H = n ? *std::max_element(height.begin(), height.end()) + 1 : 0;
    L.lvl_ptr.assign(L.H + 1, 0);
    for (int j = 0; j < n; ++j) L.lvl_ptr[height[j] + 1]++;
    for (int h = 0; h < L.H; ++h) L.lvl_ptr[h + 1] += L.lvl_ptr[h];
    L.lvl_col.assign(n, 0);
    std::vector<int> lf(L.lvl_ptr.begin(), L.lvl_ptr.end() - 1);
    for (int j = 0; j < n; ++j) L.lvl_col[lf[height[j]]++] = j;
    // From the top down, every level whose columns have at most as many slots
    // as the launch has warps (the widest level's width, or the warps of one
    // CTA per SM if fewer): every slot of its columns is a work item of its own
    // (a column without slots below the diagonal still needs its pivot: slot
    // -1), whose lanes split the slot's update terms, so that a slot costs one
    // round of loads however many terms it has; below them (wide levels of
    // short columns) a column is one item, a lane per slot.
    int widest = 1;
    for (int h = 0; h < L.H; ++h) widest = std::max(widest, L.lvl_ptr[h + 1] - L.lvl_ptr[h]);
    const long long budget = std::min<long long>(widest, (long long)slot_warps);
    auto level_items = [&](int h) {
        long long c = 0;
        for (int t = L.lvl_ptr[h]; t < L.lvl_ptr[h + 1]; ++t) {
            const int j = L.lvl_col[t];
            c += std::max(1, L.Lp[j + 1] - L.Lp[j]);
        }
        return c;
    };
    L.chain = L.H;
    while (L.chain > 0 && level_items(L.chain - 1) <= budget) --L.chain;
    // the tail for the dense phase: the longest run of columns n-1, n-2, ...
    // (closed under the tree's ancestors, like every final run) on levels at
    // most kLuTailWidth wide, at most kLuTailMax columns; none below kLuTailMin
    int T0 = n;
    while (T0 > 0 && n - T0 < kLuTailMax) {
        const int h = height[T0 - 1];
        if (L.lvl_ptr[h + 1] - L.lvl_ptr[h] > kLuTailWidth) break;
        --T0;
    }
    if (n - T0 < kLuTailMin) T0 = n;
    L.T0 = T0;
    // (the tail's items last: they wait for its whole frontier, and every item
    // waits only for items before it in the list)
    L.need.assign(n, 0);
    for (int pass = 0; pass < 2; ++pass)
        for (int h = 0; h < L.H; ++h)
            for (int t = L.lvl_ptr[h]; t < L.lvl_ptr[h + 1]; ++t) {
                const int j = L.lvl_col[t];
                if ((j >= T0) != (pass == 1)) continue;
                if (h < L.chain && j < T0) {
                    L.fitems.push_back(make_int2(j, -2));
                } else {
                    if (L.Lp[j + 1] == L.Lp[j]) L.fitems.push_back(make_int2(j, -1));
                    for (int p = L.Lp[j]; p < L.Lp[j + 1]; ++p) L.fitems.push_back(make_int2(j, p));
                }
                L.need[j] = h < L.chain && j < T0 ? 1 : std::max(1, L.Lp[j + 1] - L.Lp[j]);
            }
    // the elimination tree's children (CSR) and parents
    L.parent = parent;
    // (outside the tail; the tail's columns wait for its frontier, the columns
    // outside it whose parent is in it, listed after the children)
    L.cptr.assign(n + 1, 0);
    for (int j = 0; j < n; ++j)
        if (parent[j] >= 0 && parent[j] < T0) L.cptr[parent[j] + 1]++;
    for (int j = 0; j < n; ++j) L.cptr[j + 1] += L.cptr[j];
    L.cidx.assign(L.cptr[n], 0);
    {
        std::vector<int> cf(L.cptr.begin(), L.cptr.end() - 1);
        for (int j = 0; j < n; ++j)
            if (parent[j] >= 0 && parent[j] < T0) L.cidx[cf[parent[j]]++] = j;
    }
    L.fr0 = (int)L.cidx.size();
    for (int j = 0; j < T0; ++j)
        if (parent[j] >= T0) L.cidx.push_back(j);
    L.fr1 = (int)L.cidx.size();
    if (L.cidx.empty()) L.cidx.push_back(0);
    // the backward solve's columns outside the tail from the highest level down
    L.bcols.reserve(n);
    for (int h = L.H - 1; h >= 0; --h)
        for (int t = L.lvl_ptr[h]; t < L.lvl_ptr[h + 1]; ++t)
            if (L.lvl_col[t] < T0) L.bcols.push_back(L.lvl_col[t]);
    // every entry of J_r (CSC order) to its factor slot: 4 slot + {0: L, 1: U, 2: diagonal}
    const int nnzA = colptr[n];
    L.amap.assign(nnzA, 0);
    const auto &pos = slot_of;
    for (int c = 0; c < n; ++c)
        for (int p = colptr[c]; p < colptr[c + 1]; ++p) {
            const int i = iperm[rowidx[p]], j = iperm[c];
            if (i == j)
                L.amap[p] = 4 * j + 2;
            else if (i > j)
                L.amap[p] = 4 * pos(j, i) + 0;
            else
                L.amap[p] = 4 * pos(i, j) + 1;
        }
    return PF_OK;
}

// Upload the plan of the grid's current bus types and size its workspace.
pf_status lu_prepare(Grid *g, cudaStream_t s)
{
    if (g->lu_ready) return PF_OK;
    HostLu L;
    // the warps of one CTA per SM: an upper bound of the launch's warps
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return cuda_error(cudaGetLastError(), "jac_reduced_solve: device attributes");
    if (pf_status st = host_lu(g->nb, g->red_n, g->red_npvpq, g->red_h_colptr, g->red_h_rowidx, g->red_h_fmap,
                               std::max(1, nsm) * (kLuThreads / 32), L))
        return st;
    const size_t nnzL = (size_t)L.Lp[L.n];
    auto up = [&](int **dst, const std::vector<int> &v) -> cudaError_t {
        cudaError_t e = g->arena.alloc(dst, std::max<size_t>(v.size(), 1));
        if (e == cudaSuccess && !v.empty())
            e = cudaMemcpyAsync(*dst, v.data(), v.size() * sizeof(int), cudaMemcpyHostToDevice, s);
        return e;
    };
    cudaError_t e;
    if ((e = up(&g->lu_Lp, L.Lp)) || (e = up(&g->lu_Li, L.Li)) || (e = up(&g->lu_Rp, L.Rp)) ||
        (e = up(&g->lu_Rk, L.Rk)) || (e = up(&g->lu_Rq, L.Rq)) || (e = up(&g->lu_lvl_ptr, L.lvl_ptr)) ||
        (e = up(&g->lu_lvl_col, L.lvl_col)) || (e = up(&g->lu_perm, L.perm)) || (e = up(&g->lu_amap, L.amap)) ||
        (e = up(&g->lu_gptr, L.gptr)) || (e = up(&g->lu_need, L.need)) || (e = up(&g->lu_cptr, L.cptr)) ||
        (e = up(&g->lu_cidx, L.cidx)) || (e = up(&g->lu_parent, L.parent)) || (e = up(&g->lu_bcols, L.bcols)) ||
        (e = g->arena.alloc(&g->lu_done, 2 * (size_t)L.n + 2)) ||
        (e = g->arena.alloc(&g->lu_fitems, std::max<size_t>(L.fitems.size(), 1))) ||
        (!L.fitems.empty() && (e = cudaMemcpyAsync(g->lu_fitems, L.fitems.data(), L.fitems.size() * sizeof(int2),
                                                   cudaMemcpyHostToDevice, s))) ||
        (e = g->arena.alloc(&g->lu_gsrc, std::max<size_t>(L.gsrc.size(), 1))) ||
        (!L.gsrc.empty() && (e = cudaMemcpyAsync(g->lu_gsrc, L.gsrc.data(), L.gsrc.size() * sizeof(int2),
                                                 cudaMemcpyHostToDevice, s))) ||
        (e = g->arena.alloc(&g->lu_Lx, std::max<size_t>(nnzL, 1))) ||
        (e = g->arena.alloc(&g->lu_Ux, std::max<size_t>(nnzL, 1))) ||
        (e = g->arena.alloc(&g->lu_D, std::max(2 * L.n, 1))) || (e = g->arena.alloc(&g->lu_y, std::max(L.n, 1))) ||
        (e = cudaStreamSynchronize(s)))
        return cuda_error(e, "jac_reduced_solve: set-up");
    g->lu_n = L.n;
    g->lu_H = L.H;
    g->lu_chain = L.chain;
    g->lu_nfitems = (int)L.fitems.size();
    g->lu_nbcols = (int)L.bcols.size();
    g->lu_T0 = L.T0;
    g->lu_LpT0 = L.Lp[L.T0];
    g->lu_fr0 = L.fr0;
    g->lu_fr1 = L.fr1;
    g->lu_widest = 1;
    for (int h = 0; h < L.H; ++h) g->lu_widest = std::max(g->lu_widest, L.lvl_ptr[h + 1] - L.lvl_ptr[h]);
    g->lu_nnzL = (long long)nnzL;
    g->lu_ready = 1;
    return PF_OK;
}

void lu_release(Grid *g)
{
    for (void *p : {(void *)g->lu_Lp, (void *)g->lu_Li, (void *)g->lu_Rp, (void *)g->lu_Rk, (void *)g->lu_Rq,
                    (void *)g->lu_lvl_ptr, (void *)g->lu_lvl_col, (void *)g->lu_perm, (void *)g->lu_amap,
                    (void *)g->lu_Lx, (void *)g->lu_Ux, (void *)g->lu_D, (void *)g->lu_y, (void *)g->lu_gptr,
                    (void *)g->lu_gsrc, (void *)g->lu_need, (void *)g->lu_cptr, (void *)g->lu_cidx,
                    (void *)g->lu_parent, (void *)g->lu_bcols, (void *)g->lu_done, (void *)g->lu_fitems})
        g->arena.release(p);
    g->lu_Lp = g->lu_Li = g->lu_Rp = g->lu_Rk = g->lu_Rq = g->lu_lvl_ptr = g->lu_lvl_col = g->lu_perm = g->lu_amap =
        g->lu_gptr = nullptr;
    g->lu_need = g->lu_cptr = g->lu_cidx = g->lu_parent = g->lu_bcols = g->lu_done = nullptr;
    g->lu_gsrc = g->lu_fitems = nullptr;
    g->lu_Lx = g->lu_Ux = g->lu_D = g->lu_y = nullptr;
    g->lu_ready = 0;
}

cudaError_t launch_lu_solve(Grid *g, const double *Jr, const double *F, double *dx, cudaStream_t s)
{
    if (g->lu_n == 0) return cudaSuccess;
    LuArgs a{};
    a.n = g->lu_n;
    a.nnzA = (int)g->red_nnz;
    a.nfitems = g->lu_nfitems;
    a.nbcols = g->lu_nbcols;
    a.T0 = g->lu_T0;
    a.LpT0 = g->lu_LpT0;
    a.fr0 = g->lu_fr0;
    a.fr1 = g->lu_fr1;
    a.Lp = g->lu_Lp;
    a.Li = g->lu_Li;
    a.Rp = g->lu_Rp;
    a.Rk = g->lu_Rk;
    a.Rq = g->lu_Rq;
    a.perm = g->lu_perm;
    a.amap = g->lu_amap;
    a.gptr = g->lu_gptr;
    a.gsrc = g->lu_gsrc;
    a.need = g->lu_need;
    a.cptr = g->lu_cptr;
    a.cidx = g->lu_cidx;
    a.parent = g->lu_parent;
    a.bcols = g->lu_bcols;
    a.fitems = g->lu_fitems;
    a.done = g->lu_done;
    a.A = Jr;
    a.F = F;
    a.Lx = g->lu_Lx;
    a.Ux = g->lu_Ux;
    a.D = g->lu_D;
    a.piv = g->lu_D + g->lu_n;
    a.y = g->lu_y;
    a.dx = dx;
    a.bar = g->bar;
    a.err = g->err;
    if (g->lu_resident == 0) {
        int per_sm = 0, dev = 0, nsm = 0;
        cudaError_t e;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_lu_solve, kLuThreads, 0)) ||
            (e = cudaGetDevice(&dev)) || (e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)))
            return e;
        // one CTA per SM at most: the widest levels have a few thousand columns,
        // and more CTAs make every grid barrier dearer
        g->lu_resident = std::max(1, std::min(per_sm, 1) * nsm);
    }
    // a warp per column of the widest level (the leaves) at most
    const int ctas = std::max(1, (g->lu_widest + kLuThreads / 32 - 1) / (kLuThreads / 32));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)std::max(1, std::min(g->lu_resident, ctas)));
    cfg.blockDim = dim3(kLuThreads);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (a.T0 >= a.n) {   // no tail: one launch
        a.mode = 0;
        return cudaLaunchKernelEx(&cfg, k_lu_solve, a);
    }
    // the factorization outside the tail and the tail's outside terms; the
    // tail by one cluster; the backward solve outside the tail
    a.mode = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, k_lu_solve, a);
    if (e != cudaSuccess) return e;
    const size_t tsm = lu_tail_smem(a.n - a.T0);
    if ((e = ensure_dyn_smem(reinterpret_cast<const void *>(k_lu_tail), tsm))) return e;
    k_lu_tail<<<kLuTailCtas, kLuTailThreads, tsm, s>>>(a);
    if ((e = cudaGetLastError())) return e;
    a.mode = 2;
    return cudaLaunchKernelEx(&cfg, k_lu_solve, a);
}

}  // namespace pf

using namespace pf;

PF_API pf_status jac_reduced_solve(pf_grid *grid, const double *Jr, const double *F, double *dx, pf_stream stream)
{
    if (!grid) return set_error(PF_EINVAL, "jac_reduced_solve: grid is NULL");
    Grid *g = &grid->g;
    if (!g->red_set) return set_error(PF_EINVAL, "jac_reduced_solve: call grid_set_bus_types first");
    if (g->red_n == 0) return PF_OK;
    if (!Jr || !F || !dx) return set_error(PF_EINVAL, "jac_reduced_solve: NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    if (pf_status st = lu_prepare(g, s)) return st;
    TraceScope t(g, PF_K_LU, s);
    PF_CUDA(launch_lu_solve(g, Jr, F, dx, s));
    return PF_OK;
}
