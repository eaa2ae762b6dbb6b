// pf_internal.h - internal structures of libpfgrid (not part of the ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <atomic>
#include <vector>

#include "isincos.cuh"
#include "pfgrid.h"

#define PF_API extern "C" __attribute__((visibility("default")))

namespace pf {

// --------------------------------------------------------------- errors --
pf_status set_error(pf_status s, const char *fmt, ...);
pf_status cuda_error(cudaError_t e, const char *what);
// Raise the kernel's dynamic shared-memory limit on the current device to at
// least `bytes` (never lowers it; thread-safe).
cudaError_t ensure_dyn_smem(const void *kernel, size_t bytes);
#define PF_CUDA(call)                                            \
    do {                                                         \
        cudaError_t e_ = (call);                                 \
        if (e_ != cudaSuccess) return pf::cuda_error(e_, #call); \
    } while (0)

// device error word codes (written by kernels, read by grid_check_error)
enum : int { DEV_OK = 0, DEV_TIMEOUT = 1, DEV_BADINDEX = 2, DEV_SINGULAR = 3 };

// ------------------------------------------------- device buffer owner --
// Test hook (pf_debug_fail_allocations): when >= 0, the number of device
// allocations that still succeed before every later one fails.
extern std::atomic<int> g_alloc_countdown;

// Every buffer gets 64 bytes of slack so vector loads of the last element
// never leave the allocation.
struct DevArena {
    std::vector<void *> ptrs;
    template <class T>
    cudaError_t alloc(T **p, size_t n)
    {
        int c = g_alloc_countdown.load();
        while (c >= 0 && !g_alloc_countdown.compare_exchange_weak(c, c > 0 ? c - 1 : 0)) {
        }
        if (c == 0) return cudaErrorMemoryAllocation;   // simulated failure (test hook)
        void *q = nullptr;
        cudaError_t e = cudaMalloc(&q, n * sizeof(T) + 64);
        if (e == cudaSuccess) {
            ptrs.push_back(q);
            *p = static_cast<T *>(q);
        }
        return e;
    }
    void release(void *p);
    void free_all();
};

// K double buffers from the arena, all or none: on failure the ones already
// made are released and *out stays untouched.
template <size_t K>
inline cudaError_t alloc_all(DevArena &a, double **const (&out)[K], const size_t (&n)[K])
{
    double *b[K] = {};
    for (size_t k = 0; k < K; ++k) {
        cudaError_t e = a.alloc(&b[k], n[k]);
        if (e != cudaSuccess) {
            for (size_t q = 0; q < k; ++q) a.release(b[q]);
            return e;
        }
    }
    for (size_t k = 0; k < K; ++k) *out[k] = b[k];
    return cudaSuccess;
}

// ------------------------------------------------ host index structures --
// Topology-only structures, built once on the host (host_layout.cpp).
enum : int { EW_ACCUM = 0x40000000, EW_KMASK = 0x3fffffff };

struct HostTopo {
    int nb = 0, nl = 0, nnz = 0;
    std::vector<int> from, to;
    std::vector<int> tp;        // [nb+1] terminals of bus i: sorted positions tp[i] .. tp[i+1]
    std::vector<int> tsort;     // [2nl] terminal ids sorted by (owner, other, branch)
    std::vector<int> tpos;      // [2nl] sorted position of terminal t
    std::vector<int> tkpos;     // [2nl] position of the other bus in the owner's Ybus row
    std::vector<int> taccum;    // [2nl] 1 if not the first terminal of its (owner, other) run
    std::vector<int2> tnbr;     // [2nl] by sorted position: {other bus, kpos | EW_ACCUM}
    std::vector<int> town;      // [2nl] by sorted position: owner bus
    std::vector<int> tmir;      // [2nl] by sorted position: sorted position of the other end's terminal
    std::vector<int> rp, ci;    // Ybus CSR pattern
    std::vector<int> ybeg, yend, ydiag;  // per nnz: sorted-terminal stamp range; row if diagonal else -1
    std::vector<int> kd;        // [nb] position of the diagonal in row i
    std::vector<int> jrp, jci;  // canonical J pattern
    int owner(int t) const { return (t & 1) ? to[t >> 1] : from[t >> 1]; }
    int other(int t) const { return (t & 1) ? from[t >> 1] : to[t >> 1]; }
};

// Element-wise windows: consecutive bus ranges whose terminals (contiguous in
// sorted order) are evaluated one per thread by one CTA of `tb` threads; a
// window holds at most tb buses and at most tb terminals (a single bus with
// more terminals gets a window of its own and its terminals are looped over).
struct HostEw {
    int tb = 0, nwin = 0;
    int tfac = 1;       // at most tfac * tb terminals per window (threads loop over them)
    int max_L = 0;      // max over windows of 2 * (Ybus nnz of the window's rows)
    int max_nt = 0;     // max terminals in a window
    int max_nbus = 0;   // max buses in a window
    int max_nh = 0;     // max ghost buses of a window
    int max_nph = 0;    // max phasor slots (own + ghost buses) of a window
    std::vector<int> win_bus;   // [nwin+1]
    // Ghost buses: the buses outside a window that its terminals reach,
    // sorted, window w's at hbus[hptr[w] .. hptr[w+1]).  A window's phasor
    // table holds its own buses (slots 0 .. nbus-1) then its ghost buses.
    std::vector<int> hptr, hbus;
    // per sorted terminal: {phasor-table slot of the other bus, Ybus slot
    // position | EW_ACCUM} (tnbr with the bus replaced by its window slot)
    std::vector<int2> tloc;
    // per window w: desc[2w] = {first bus, buses, first terminal, terminals},
    // desc[2w+1] = {first Ybus row entry, J slice length, phasor slots, 0};
    // slotbus[w * max_nph + j] = bus of phasor slot j
    std::vector<int4> desc;
    std::vector<int> slotbus;
    // per bus o of window w: {2 (rowptr[o] - rowptr[b0]) (its row in the
    // window's J slice), Ybus row length, diagonal position, tp[o] - tp[b0]}
    std::vector<int4> bmeta;
    // per window, its buses (window-local) by decreasing terminal count (ties
    // in bus order) at rorder[b0 ...]: the reduction's thread-to-bus map, so
    // that the lanes of a warp loop over about as many terminals
    std::vector<int> rorder;
};

pf_status host_topology(int nb, int nl, const int *from, const int *to, HostTopo &H);
// Windows of consecutive buses (<= tb buses, <= tfac * tb terminals).  With
// target_nwin > 0 they are cut at equal estimated cost into at most
// target_nwin windows when the plain greedy cut gives fewer.
pf_status host_ew(const HostTopo &H, int tb, HostEw &E, int tfac = 1, int target_nwin = 0);
pf_status host_selfcheck(const HostTopo &H, const HostEw &E);
// Per window, the branches whose from-terminal lies in it: {window-local
// terminal, branch} at brl[w * max_nbr + j], j < nbr[w] (every branch once).
pf_status host_window_branches(const HostTopo &H, const HostEw &E, std::vector<int2> &brl, std::vector<int> &nbr,
                               int &max_nbr);

// Shared-memory plan of the element-wise kernels (byte offsets, 16-aligned):
//   bm  int4    [max_nbus]   per bus {J-slice row offset, row length, diagonal position, first terminal}
//   yd  double2 [max_nbus]   per bus self sum
//   kg  double2 [2 max_nt]   per terminal K and G (injection kernel: K only)
//   kp  int     [max_nt]     per terminal slot position | EW_ACCUM (Jacobian kernel)
//   jst double  [2 max_L]    the window's J slice (P half, then Q half)
//   pq  double  [2 pqs]      P then Q of the window, parity-aligned with global memory
//   ph                       phasor table (below)
//   ord int     [max_nbus]   the reduction's thread-to-bus map (HostEw::rorder)      (max_nph > 0)
//   w2  double2 [max_nbus]   (v^2, 2 v) of the window's own buses                     (max_nph > 0)
struct EwSmem {
    uint32_t bm, yd, kg, kp, jst, pq, pqs, ph, ord, w2, total;
};
// max_nph > 0 (the single-evaluation kernel) adds a phasor table of that many
// slots: V of the own buses in block floating point and 2^62 (cos, sin), each
// a pair of 64-bit integers, and (v, 1/v), and the ord and w2 arrays
__host__ __device__ inline EwSmem ew_smem_plan(int max_nbus, int max_nt, int max_L, bool jac, int max_nph = 0)
{
    EwSmem p;
    p.pqs = ((uint32_t)max_nbus + 3u) & ~1u;   // even, >= max_nbus + 2
    p.bm = 0;
    p.yd = p.bm + 16u * (uint32_t)max_nbus;
    p.kg = p.yd + 16u * (uint32_t)max_nbus;
    p.kp = p.kg + (jac ? 32u : 16u) * (uint32_t)max_nt;
    p.jst = p.kp + (jac ? ((4u * (uint32_t)max_nt + 15u) & ~15u) : 0u);
    p.pq = p.jst + (jac ? 16u * (uint32_t)max_L : 0u);
    p.ph = p.pq + 16u * p.pqs;
    p.ord = p.ph + 48u * (uint32_t)max_nph;
    p.w2 = p.ord + (max_nph > 0 ? (4u * (uint32_t)max_nbus + 15u) & ~15u : 0u);
    p.total = p.w2 + (max_nph > 0 ? 16u * (uint32_t)max_nbus : 0u);
    return p;
}
constexpr uint32_t kMaxSmem = 227u * 1024u;
constexpr int kYbusRowChunk = 256;
// shared memory of the (cos, sin) table every phasor-forming CTA holds
constexpr uint32_t kTrigSmem = kITrigN * (uint32_t)sizeof(ITrig);
// words of the batched kernels' grid-barrier state: parity, two counters on their
// own lines, and the loss total's arrival count (k_batched.cu) on a fourth
constexpr int kBarWords = 128;
constexpr int kLossCountWord = 96;

// Shared memory of the small-batch adjoint (k_adj1, one item per CTA): bus
// metadata and self sums, both flows of every terminal and its two phasor
// slots, loss / gradient staging, the phasor (as doubles and in the fixed-point
// form), residual and bus-name tables of the own and ghost slots, (v, 1/v) of
// the own buses, the sine/cosine table.
struct Adj1Smem {
    uint32_t bm, yd, K, M, loc, pq, V, R, W, uf, af, vs, slot, tab, total, pqs;
};
__host__ __device__ inline Adj1Smem adj1_smem_plan(int max_nbus, int max_nt, int max_nph)
{
    Adj1Smem p;
    const uint32_t nbus = (uint32_t)max_nbus, nt = (uint32_t)max_nt, nph = (uint32_t)max_nph;
    p.pqs = (nbus + 3u) & ~1u;   // even, >= max_nbus + 2
    p.bm = 0;
    p.yd = p.bm + 16u * nbus;
    p.K = p.yd + 16u * nbus;
    p.M = p.K + 16u * nt;
    p.loc = p.M + 16u * nt;
    p.pq = p.loc + ((8u * nt + 15u) & ~15u);
    p.V = p.pq + 16u * p.pqs;
    p.R = p.V + 16u * nph;
    p.W = p.R + 16u * nph;
    p.uf = p.W + 16u * nbus;   // per slot: 2^62 (cos, sin), V in block floating point, v (fixrot.cuh)
    p.af = p.uf + 16u * nph;
    p.vs = p.af + 16u * nph;
    p.slot = p.vs + 8u * ((nph + 1u) & ~1u);
    p.tab = p.slot + ((4u * nph + 15u) & ~15u);
    p.total = p.tab + kTrigSmem;
    return p;
}
// threads per CTA of k_adj1
constexpr int kAdj1Threads = 512;

// ------------------------------------------------ device-side structure --
struct EwDev {
    int tb = 0, nwin = 0, max_L = 0, max_nt = 0, max_nbus = 0, max_nph = 0;
    int4 *desc = nullptr;     // [2 nwin] window descriptors (HostEw::desc)
    int *slotbus = nullptr;   // [nwin * max_nph] bus of every phasor slot
    int4 *bmeta = nullptr;    // [nb] window-relative bus metadata (HostEw::bmeta)
    int *rorder = nullptr;    // [nb] the reduction's thread-to-bus map (HostEw::rorder)
    int2 *tloc = nullptr;     // [T] {phasor slot of the other bus, slot position | flags}
};

struct Grid {
    int nb = 0, nl = 0, nnz = 0;
    pf_config cfg{};
    DevArena arena;
    HostTopo topo;
    // Ybus (device)
    int *rp = nullptr, *ci = nullptr;
    // the Ybus row kernels' thread-to-row map: each chunk of kYbusRowChunk rows
    // by decreasing length (ties in row order), so a warp's rows take equally
    // many loop trips and FP64 warp instructions keep their lanes busy
    int *yrow = nullptr;
    double2 *yv = nullptr;
    // the Ybus values in block floating point (fixrot.cuh): yfx 2^(yce - 1085),
    // yce = 0 where a value is not representable (the kernels then take yv)
    longlong2 *yfx = nullptr;
    int *yce = nullptr;
    int *ybeg = nullptr, *yend = nullptr, *ydiag = nullptr;
    int *kd = nullptr;                     // [nb] diagonal position per row
    // J pattern (device)
    int *jrp = nullptr, *jci = nullptr;
    // terminals in sorted order (device)
    int *tp = nullptr;                     // [nb+1]
    double2 *tself = nullptr, *tcoup = nullptr;
    // Yc in block floating point (fixrot.cuh): tcfx 2^(tce - 1085), tce = 0 where
    // it is not representable (the kernels then take tcoup)
    longlong2 *tcfx = nullptr;
    int *tce = nullptr;
    int2 *br_hk = nullptr;                 // [nl] end buses (from, to) of branch l
    double4_32a *br_aux = nullptr;         // [nl] {1/m, cos phi, sin phi, -(b + b_sh/2)} of branch l (with the constants)
    int2 *tnbr = nullptr;                  // {other bus, kpos | EW_ACCUM}
    int *town = nullptr;                   // owner bus
    int *tpos = nullptr;                   // [2nl] sorted position of terminal t
    double2 *bus_ysh = nullptr;            // [nb]
    double2 *bus_yd = nullptr;             // [nb] bus shunt + sum of the bus's terminal self constants
    EwDev ew;
    uint32_t ew_smem_jac = 0, ew_smem_inj = 0, ew_smem_host = 0, ew_smem_red = 0;   // dynamic shared memory the kernels are configured for
    int nsm = 0;                                  // SM count (cached)
    int *tmir = nullptr;                   // [2nl] by sorted position: sorted position of the mirror terminal
    // device copies of the current parameters (branch gradients need them)
    double *p_g = nullptr, *p_b = nullptr, *p_bsh = nullptr, *p_tap = nullptr, *p_shift = nullptr;
    unsigned int *bar = nullptr;   // [kBarWords] grid-barrier state of the batched kernels (ptx.cuh)
    // per-call workspace of the Ybus method's phasor step (device)
    double4_32a *ph_u = nullptr;   // [nb] {cos, sin, v, 1/v}
    double2 *ph_v = nullptr;       // [nb] V = v e^{j theta}
    int *err = nullptr;            // device error word
    // the two-step study path (k_study.cu): K_t, G_t of every sorted terminal
    double4_32a *ts_KG = nullptr;
    double *vs_V = nullptr;   // [2 nb] voltages of the storage-layout study (inj_ybus_study)
    // eval_host staging (lazy)
    double *st_vm = nullptr, *st_va = nullptr, *st_P = nullptr, *st_Q = nullptr, *st_J = nullptr;
    // reduced Newton Jacobian (grid_set_bus_types): CSC pattern, the canonical J
    // position of every reduced entry, the bus of every mismatch entry, and
    // scratch for the full evaluation it is gathered from
    int red_set = 0, red_n = 0, red_npvpq = 0;
    long long red_nnz = 0;
    int *red_colptr = nullptr, *red_rowidx = nullptr, *red_jmap = nullptr, *red_fmap = nullptr;
    // inverse maps for the fused element-wise path: the reduced (CSC) index of
    // every canonical J position, and of every bus's P and Q equation (-1: not kept)
    int *red_jinv = nullptr;
    int2 *red_binv = nullptr;
    // a caller's Jacobian pattern (jac_set_target_pattern, Alg. 2): the
    // position in it of every canonical entry, and scratch for the Ybus method
    int tgt_set = 0;
    long long tgt_nnz = 0;
    int *tgt_map = nullptr;
    double *tgt_J = nullptr;
    double *red_P = nullptr, *red_Q = nullptr, *red_J = nullptr;
    // host copies of the reduced pattern (the LU analysis reads them)
    std::vector<int> red_h_colptr, red_h_rowidx, red_h_fmap;
    // Newton-Raphson workspace (powerflow_newton): F, J_r (CSC), step, max |F|
    double *nt_F = nullptr, *nt_J = nullptr, *nt_dx = nullptr;
    unsigned long long *nt_max = nullptr;
    // sparse LU of the reduced system (lu.cu): plan of the current bus types
    // (CSC of L's pattern, row structures, levels, permutation, value map) and
    // the factor storage
    int lu_ready = 0, lu_n = 0, lu_H = 0, lu_chain = 0, lu_resident = 0, lu_widest = 0;
    long long lu_nnzL = 0;
    int *lu_Lp = nullptr, *lu_Li = nullptr, *lu_Rp = nullptr, *lu_Rk = nullptr, *lu_Rq = nullptr;
    int *lu_lvl_ptr = nullptr, *lu_lvl_col = nullptr, *lu_perm = nullptr, *lu_amap = nullptr, *lu_gptr = nullptr;
    int *lu_need = nullptr, *lu_cptr = nullptr, *lu_cidx = nullptr, *lu_parent = nullptr, *lu_bcols = nullptr;
    int *lu_done = nullptr;   // [2n + 1] per column: finished factorization items, backward solve done; the item counter
    int lu_nfitems = 0, lu_nbcols = 0, lu_T0 = 0, lu_LpT0 = 0;   // items; the tail's first column and slot
    int lu_fr0 = 0, lu_fr1 = 0;                                  // the tail's frontier in lu_cidx
    int2 *lu_gsrc = nullptr, *lu_fitems = nullptr;
    double *lu_Lx = nullptr, *lu_Ux = nullptr, *lu_D = nullptr, *lu_y = nullptr;
    // tracer: events [2 * capacity], kernel id per record
    std::vector<cudaEvent_t> tr_ev;
    std::vector<int> tr_kernel;
    int tr_n = 0;
};

// Brackets one kernel launch with tracer events when tracing is on.
struct TraceScope {
    Grid *g;
    int slot;
    cudaStream_t s;
    TraceScope(Grid *g_, int kernel, cudaStream_t s_) : g(g_), slot(-1), s(s_)
    {
        if (!g->tr_ev.empty() && g->tr_n < (int)g->tr_kernel.size()) {
            slot = g->tr_n++;
            g->tr_kernel[slot] = kernel;
            cudaEventRecord(g->tr_ev[2 * slot], s);
        }
    }
    ~TraceScope()
    {
        if (slot >= 0) cudaEventRecord(g->tr_ev[2 * slot + 1], s);
    }
};

// Launch with cudaLaunchKernelEx; `pdl` allows programmatic dependent launch
// (the kernel may start while the preceding kernel in the stream finishes and
// must call griddepcontrol.wait before reading that kernel's results).
template <typename... KArgs, typename... Args>
inline cudaError_t launch_k(void (*kernel)(KArgs...), int grid, int block, size_t smem, cudaStream_t s, bool pdl,
                            Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// kernel launchers (k_*.cu); each returns the status of its launch(es)
cudaError_t launch_branch_constants(Grid *g, const double *gg, const double *gb, const double *gbsh,
                                    const double *gtap, const double *gshift, cudaStream_t s);
cudaError_t launch_ybus_values(Grid *g, const double *gs, const double *bs, cudaStream_t s);
cudaError_t ensure_trig_table();   // once per device, synchronous
const ITrig *trig_table();         // device address of the (cos, sin) table of isincos.cuh
cudaError_t launch_phasor(int nb, const double *vm, const double *va, double4_32a *U, double2 *V, cudaStream_t s);
cudaError_t launch_phasor_fix(int nb, const double *vm, const double *va, double4_32a *U, cudaStream_t s);
struct ScenOut;
cudaError_t launch_ybus_rows(const Grid *g, int S, bool out, const ScenOut *sc, const long long *joff,
                             const double4_32a *U, bool jac, double *P, double *Q, double *J, int lanes, int blk,
                             cudaStream_t s);
// the Ybus method with the phasor step fused into the row kernel (one launch)
cudaError_t launch_ybus_fused(const Grid *g, bool jac, const double *vm, const double *va, double *P, double *Q,
                              double *J, cudaStream_t s);
// element-wise: one CTA per window (phasors of its own and ghost buses, evaluation, reduction)
cudaError_t ew_blocks_per_sm(int tb, size_t smem, int *per_sm);   // CTAs of k_ew<true> that fit on one SM
cudaError_t launch_inj_ew(Grid *g, const double *vm, const double *va, double *P, double *Q, cudaStream_t s);
cudaError_t launch_jac_ew(Grid *g, const double *vm, const double *va, double *P, double *Q, double *J,
                          cudaStream_t s, bool host_out = false);   // host_out: P, Q, J in mapped host memory
// the Jacobian evaluation with the reduced Newton system (F, CSC values) as its only output
cudaError_t launch_jac_ew_reduced(Grid *g, const double *vm, const double *va, const double *Ps, const double *Qs,
                                  double *F, double *Jr, cudaStream_t s);
// the Jacobian evaluation with J stored through map (canonical position -> Jt
// position), P and Q (may be NULL) stored as usual
cudaError_t launch_jac_ew_mapped(Grid *g, const double *vm, const double *va, double *P, double *Q, const int *map,
                                 double *Jt, cudaStream_t s);

// reduced Newton system (reduced.cu)
cudaError_t launch_reduce(Grid *g, const int *map, const double *Pspec, const double *Qspec, double *F, double *Jr,
                          cudaStream_t s);

// sparse LU of the reduced system (lu.cu): the host analysis of a reduced
// pattern (permutation new -> reduced index, CSC of L's pattern, per column the
// (k, position of L(j, k)) pairs of its row, columns by tree height, the top
// levels narrow enough for one CTA from `chain` on, and each reduced entry's
// factor slot 4 slot + {0 L, 1 U, 2 diagonal}), its upload, and the solve
struct HostLu {
    int n = 0, H = 0, chain = 0;
    int T0 = 0;             // the tail (columns T0 .. n-1) factored as a dense block; n: none
    int fr0 = 0, fr1 = 0;   // the tail's frontier (the columns outside it whose parent is in it) in cidx
    std::vector<int> perm, Lp, Li, Rp, Rk, Rq, lvl_ptr, lvl_col, amap;
    std::vector<int> gptr;    // [nnzL + 1] update terms of every factor slot
    std::vector<int2> gsrc;   // {slot of L(i, k), slot of L(j, k)}, k ascending per slot
    // dependency-driven schedule: the factorization's work items in level order
    // ({column, -2}: the whole column by one warp; {column, slot or -1}: one slot
    // of a column of the narrow top), the items of every column, the columns'
    // children in the elimination tree (CSR) and parents, and the columns of the
    // backward solve from the root down
    std::vector<int2> fitems;
    std::vector<int> need, cptr, cidx, parent, bcols;
};
pf_status host_lu(int nb, int n, int npvpq, const std::vector<int> &colptr, const std::vector<int> &rowidx,
                  const std::vector<int> &fmap, int slot_warps, HostLu &L);
pf_status lu_prepare(Grid *g, cudaStream_t s);
void lu_release(Grid *g);
cudaError_t launch_lu_solve(Grid *g, const double *Jr, const double *F, double *dx, cudaStream_t s);

// ----------------------------------------------------------- batches ----
// S scenarios over one grid: per-scenario voltage states and an optional N-1
// outage (one branch removed).  Scenario s's Jacobian is stored on its own
// pattern (the base pattern without the outage's off-diagonal pair when no
// parallel branch keeps it) at J + joff[s].
struct ScenOut {
    int h, k;          // outage branch end buses (-1: none)
    int ph, pk;        // sorted positions of its two terminals
    int del;           // 1 if the (h, k) / (k, h) Ybus entries disappear
    int kh, kk;        // positions of k in row h and of h in row k (base pattern)
    int l;             // outage branch (-1: none)
};

struct Batch {
    Grid *g = nullptr;
    int S = 0;
    int nsm = 0;                     // SMs of the device the batch was made on
    int has_outage = 0;              // some scenario removes a branch
    pf_batch_config cfg{};           // launch configuration (batch_set_config, batch_autotune)
    DevArena arena;
    std::vector<ScenOut> h_sc;
    std::vector<long long> h_joff;   // [S+1]
    ScenOut *sc = nullptr;           // [S]
    long long *joff = nullptr;       // [S+1]
    double4_32a *U = nullptr;        // [S][nb]
    double2 *V = nullptr;            // [S][nb]
    double2 *r = nullptr;            // [S][nb] loss residual (2 wP dP, 2 wQ dQ)
    double *lpart = nullptr;         // [S][nwin] per-window loss partial sums
    double *lscen = nullptr;         // [S] per-scenario losses when the caller wants only their total
    // co-resident CTAs of the batched kernels (inj, jac, adjoint, k_adj1, and
    // the loss-only forms of the last two)
    int resident[6] = {0, 0, 0, 0, 0, 0};
    // the batch's own element-wise windows: throughput-bound, so every thread
    // owns a bus in the reduction and loops over up to tfac terminals
    int tb = 0, tfac = 1, nwin = 0, max_L = 0, max_nt = 0, max_nbus = 0;
    int *win_bus = nullptr;          // [nwin+1]
    int *rorder = nullptr;           // [nb] the reductions' thread-to-bus map (HostEw::rorder)
    // small batches (about one item per SM): the adjoint runs k_adj1, one
    // item per CTA, which forms each window's phasors with its ghost buses
    // instead of a separate phase and barrier
    int ghost = 0, max_nph = 0;
    int4 *desc = nullptr;            // [2 nwin] window descriptors (HostEw::desc; desc[2w+1].w = branches of w)
    int *slotbus = nullptr;          // [nwin * max_nph]
    int2 *tloc = nullptr;            // [T]
    int max_nbr = 0;
    int2 *brl = nullptr;             // [nwin * max_nbr] the window's branches (host_window_branches)
};

// the batch's window plan for a configuration (batch.cu), its upload, and the
// tuned configuration of the batch's size class from the cache file named by
// PFGRID_TUNE_CACHE, if any (batch_tune.cu)
pf_status batch_plan(const Grid *g, int nscen, int tb, int tfac, HostEw &E, bool &ghost);
pf_status batch_upload(Batch *b, HostEw &E, bool ghost, cudaStream_t st);
pf_status batch_apply_cached(Batch *b, cudaStream_t st);
pf_status batch_apply_config(Batch *b, const pf_batch_config &c, cudaStream_t st);

cudaError_t launch_ew_batched(Batch *b, bool jac, const double *vm, const double *va, double *P, double *Q,
                              double *J, cudaStream_t s);
cudaError_t launch_ybus_batched(Batch *b, bool jac, const double *vm, const double *va, double *P, double *Q,
                                double *J, cudaStream_t s);
cudaError_t launch_adjoint(Batch *b, const double *vm, const double *va, const double *Ps, const double *Qs,
                           const double *wP, const double *wQ, const double *Lbar, double *L, double *Ltot,
                           double *gvm, double *gva, double *gg, double *gb, double *gbsh, double *gtap,
                           cudaStream_t s);
cudaError_t launch_loss(Batch *b, const double *vm, const double *va, const double *Ps, const double *Qs,
                        const double *wP, const double *wQ, double *L, double *Ltot, cudaStream_t s);

}  // namespace pf

struct pf_grid {
    pf::Grid g;
};

struct pf_batch {
    pf::Batch b;
};
