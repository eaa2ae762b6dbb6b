// k_elementwise.cu - element-wise method (Sec. II-B, IV-C) on the GPU: one
// CTA per window of consecutive buses, one launch per evaluation and no
// synchronisation between CTAs.
//
// Phasors.  The paper's element-wise loop evaluates the angle-difference terms
// inside its per-line loop; here each CTA first forms the phasors
// U = e^{j theta}, V = v U of every bus its terminals touch - its own buses
// and its ghost buses (the other ends outside the window, listed at setup) -
// into a window-local table in shared memory.  A bus is transformed once per
// window that touches it (about 1.6-1.8 times per bus on grids numbered with
// spatial locality) instead of once per terminal, and no CTA waits for
// another: the kernel is a plain launch of one CTA per window.
//
// Evaluation step (the per-element loop of Sec. IV-C, one terminal per
// thread).  Terminal t of a branch (owner bus o, other bus q) has precomputed
// constants Ys_t, Yc_t (k_setup.cu) such that its complex power (Eqs. 5-6) is
//     S_t = v_o^2 conj(Ys_t) + K_t,   K_t = conj(Yc_t) V_o conj(V_q),
// where V_o conj(V_q) = v_o v_q e^{j(theta_o - theta_q)} carries the sine and
// cosine of the angle difference.  Its 8 partials (16 per branch):
//     dS_t/dtheta_q = -j K_t            dS_t/dv_q = K_t / v_q = conj(Yc_t) V_o conj(U_q)
//     dS_t/dtheta_o = +j K_t            dS_t/dv_o = 2 v_o conj(Ys_t) + K_t / v_o
// The thread computes G = conj(Yc_t) V_o conj(U_q) (= dS_t/dv_q) in 64-bit
// fixed point on the integer pipe (fixrot.cuh: the phasor table holds U as
// 2^62-scaled integers and V_o in block floating point, the setup Yc_t), then
// K_t = v_q G: 2 FP64 instructions.  The injections alone take the same steps
// (K_t only).
//
// Reduction step (Eq. 7 and the copy-add of Fig. 2, without atomics).
// Terminals are stored sorted by (owner, other bus), so a CTA owns a window of
// consecutive buses together with all of their terminals: the off-diagonal
// slot (o, q) is written by the terminal's thread (parallel branches,
// adjacent in the sorted order, are added by the owner's thread below), and
// two threads per bus (the real and the imaginary parts; the window's buses
// taken by decreasing terminal count, so that a warp's lanes loop equally
// long) sum its terminals' K in a fixed order:
//     S_o           = v_o^2 conj(Yd_o) + sum K
//     dS_o/dtheta_o = j sum K
//     dS_o/dv_o     = 2 v_o conj(Yd_o) + (sum K) / v_o
// with Yd_o = sum_t Ys_t + y_sh,o, a parameter-only per-bus constant formed at
// setup from the same terminal constants.
//
// Work balance.  The windows are cut at equal estimated FP64 cost into a
// whole number of waves of the CTAs that fit on the GPU (host_layout.cpp), so
// every SM gets the same work.
//
// GB300 data movement.  Every global load of a window (its voltages, the
// ghost voltages, the terminal constants of the first pass, the bus metadata)
// is issued before any arithmetic, in two levels of dependent loads (the
// fixed-stride window records, then what they index).  A window's Jacobian rows are one
// contiguous slice of each of the P and Q halves of J (canonical layout): it
// is assembled in shared memory and written back with TMA bulk stores,
// together with P and Q.
#include <algorithm>

#include "fastmath.cuh"
#include "fixrot.cuh"
#include "pf_internal.h"
#include "ptx.cuh"

namespace pf {

struct EwArgs {
    int nnz, nwin, max_nbus, max_nt, max_L, max_nph, aligned;
    const int4 *desc, *bmeta;
    const int *slotbus, *town, *rorder;
    const double2 *yd, *tcoup;
    const longlong2 *tcfx;
    const int *tce;
    const ITrig *trig;
    const int2 *tloc;
    const double *vm, *va;
    double *P, *Q, *J;
    // mapped outputs (k_ew_red): the destination of every canonical J position
    // in Jr (-1: not kept) and, for the reduced Newton system, the reduced index
    // of every bus's P and Q equation
    const int *jinv;
    const int2 *binv;
    const double *Ps, *Qs;
    double *F, *Jr;
};

#ifdef PF_PHASE_PROBE
// Phase probe (builds with -DPF_PHASE_PROBE only): thread 0 of every CTA of
// the single-evaluation kernel records, per window, the %globaltimer at its
// start and end, its SM, the clock64 cycles from its start to the end of each
// phase (loads, phasors, evaluation, reduction, stores), and the %globaltimer
// when its programmatic-dependent-launch wait returned.
constexpr int kProbeMaxWin = 8192, kProbeSlots = 9;
__device__ unsigned long long g_phase_probe[kProbeMaxWin * kProbeSlots];
__device__ __forceinline__ unsigned long long probe_gtimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
#define PF_PROBE_MARK(k)                                 \
    do {                                                 \
        if (probe && tid == 0) pt[k] = clock64() - pt0;  \
    } while (0)
#else
#define PF_PROBE_MARK(k) \
    do {                 \
    } while (0)
#endif

// Write x[b0 .. b1) from shared staging `s` (element b0 at s[b0 & 1]) to
// global memory: an unaligned head and tail element by plain stores, the
// 16-byte aligned middle by one bulk store (issued by the calling thread).
__device__ __forceinline__ void store_range(double *x, const double *s, int b0, int b1)
{
    const int par = b0 & 1;
    if (par) x[b0] = s[1];
    const int ge = b0 + par;
    const int cm = (b1 - ge) & ~1;
    if (cm > 0) bulk_s2g(x + ge, s + 2 * par, 8u * (uint32_t)cm);
    if ((b1 - ge) & 1) x[b1 - 1] = s[b1 - 1 - b0 + par];
}

// One window per CTA; with PERSIST the CTAs loop over the windows
// (grid-strided), so that the first windows' outputs leave while later
// windows are evaluated (outputs in host memory, where the host link is the
// bound).
template <bool JAC, bool PERSIST, bool RED = false>
__device__ __forceinline__ void ew_windows(const EwArgs &a)
{
    extern __shared__ __align__(16) char smem[];
    const EwSmem sp = ew_smem_plan(a.max_nbus, a.max_nt, JAC ? a.max_L : 0, JAC, a.max_nph);
    int4 *sbm = reinterpret_cast<int4 *>(smem + sp.bm);
    double2 *syd = reinterpret_cast<double2 *>(smem + sp.yd);
    double2 *sSv = syd;   // the Jacobian kernels keep v^2 conj(Yd) where the others keep Yd
    double2 *skg = reinterpret_cast<double2 *>(smem + sp.kg);
    int *skp = reinterpret_cast<int *>(smem + sp.kp);
    double *jst = reinterpret_cast<double *>(smem + sp.jst);
    double *spq = reinterpret_cast<double *>(smem + sp.pq);
    longlong2 *sA = reinterpret_cast<longlong2 *>(smem + sp.ph);             // own buses: V in block floating point
    longlong2 *sU = sA + a.max_nph;                                          // 2^62 (cos, sin)
    double2 *sW = reinterpret_cast<double2 *>(sU + a.max_nph);               // (v, 1/v)
    double2 *sW2 = reinterpret_cast<double2 *>(smem + sp.w2);               // own buses: (v^2, 2 v)
    int *sord = reinterpret_cast<int *>(smem + sp.ord);                     // reduction thread -> bus
    ITrig *tab = reinterpret_cast<ITrig *>(smem + sp.total);
    const int tid = threadIdx.x, TB = blockDim.x;
    // programmatic dependent launch: the next kernel in the stream may start
    // its CTAs as these exit (it waits before it reads or writes anything
    // this kernel may still touch, see below)
    pdl_launch_dependents();
    for (int w = blockIdx.x; w < a.nwin; w += gridDim.x) {
#ifdef PF_PHASE_PROBE
        const bool probe = !PERSIST && !RED && w < kProbeMaxWin;
        const unsigned long long gt0 = probe && tid == 0 ? probe_gtimer() : 0ull;
        const long long pt0 = clock64();
        long long pt[5] = {0, 0, 0, 0, 0};
        unsigned long long gtw = 0ull;
#endif
        if (PERSIST) __syncthreads();   // the previous window's shared-memory readers are done
        // two levels of dependent loads: the window's records (descriptor, the
        // bus of the thread's first phasor slot), then everything they index
        const int *sbus = a.slotbus + (long long)w * a.max_nph;
        const int o0 = tid < a.max_nph ? sbus[tid] : 0;
        const int4 d0 = a.desc[2 * w], d1 = a.desc[2 * w + 1];
        // the sine/cosine table is requested with the first level: issued after
        // the second-level gathers it would arrive at the end of the kernel's
        // whole input burst, and every warp waits for it at the barrier below
        const bool load_tab = !PERSIST || w == (int)blockIdx.x;
        const ITrig *trig = a.trig + (blockIdx.x % kITrigCopies) * kITrigN;
        ITrig tv0 = {0ull, 0ull};
        if (load_tab && tid < kITrigN) tv0 = trig[tid];
        const int b0 = d0.x, nbus = d0.y, b1 = b0 + nbus, t0 = d0.z, nt = d0.w;
        const int r0 = d1.x, L = JAC ? d1.y : 0, nph = d1.z;

        // ---- loads of topology data (fixed when the grid's layout is built;
        // no kernel writes them): the bus thread's metadata (a window has at
        // most blockDim.x buses), kept in registers until the phasors are done
        // so its latency hides behind them, and the first terminal's slots ----
        int4 bmo = make_int4(0, 0, 0, 0);
        int ordo = 0;
        if (tid < nbus) {
            bmo = a.bmeta[b0 + tid];
            ordo = a.rorder[b0 + tid];
        }
        int2 nq = make_int2(0, 0);
        int ol = 0;
        if (tid < nt) {
            nq = a.tloc[t0 + tid];
            ol = a.town[t0 + tid];   // made window-local at first use: nothing before the
                                     // barrier below may wait for a second-level load
        }
        // ---- the previous kernel in the stream may still run (programmatic
        // dependent launch): the state, the parameter-dependent constants and
        // the outputs are read and written only after it has completed; their
        // lines are only brought into L2 before (prefetches return no data) ----
        if (tid < nph) {
            prefetch_l2(a.va + o0);
            prefetch_l2(a.vm + o0);
        }
        if (tid < nbus) prefetch_l2(a.yd + b0 + tid);
        if (tid < nt) {
            prefetch_l2(a.tcfx + t0 + tid);
            prefetch_l2(a.tce + t0 + tid);
        }
        pdl_wait();
#ifdef PF_PHASE_PROBE
        if (probe && tid == 0) gtw = probe_gtimer();
#endif
        double th = 0.0, v = 0.0;
        if (tid < nph) {
            th = a.va[o0];
            v = a.vm[o0];
        }
        double2 ydo = make_double2(0.0, 0.0);
        if (tid < nbus) ydo = a.yd[b0 + tid];
        longlong2 yf = make_longlong2(0, 0);
        int ey = 0;
        if (tid < nt) {
            yf = a.tcfx[t0 + tid];
            ey = a.tce[t0 + tid];
        }
        if (load_tab) {
            if (tid < kITrigN) tab[tid] = tv0;
            for (int k = tid + TB; k < kITrigN; k += TB) tab[k] = trig[k];
        }
        __syncthreads();
        PF_PROBE_MARK(0);

        // ---- phasor table of the window (Sec. IV-B.1 step 1, own and ghost buses) ----
        for (int j = tid; j < nph; j += TB) {
            if (j != tid) {
                const int o = sbus[j];
                th = a.va[o];
                v = a.vm[o];
            }
            int64_t C, S;
            int_sincos_q62(th, tab, &C, &S);
            sU[j] = make_longlong2(C, S);
            double iv = 0.0;
            if (j < nbus) {
                int64_t ar, ai;
                fix_phasor(C, S, v, &ar, &ai);
                sA[j] = make_longlong2(ar, ai);
            }
            if (JAC) {
                // 1/v is read for the window's own buses only: warps of ghost
                // slots skip it (a warp-uniform branch), mixed warps form it
                // for all lanes; and the parameter-and-magnitude terms of the
                // reduction, 2 v conj(Yd) and v^2 conj(Yd), formed once per bus
                // here (where the FP64 pipe is idle) instead of by both threads
                // of its pair (slot j < nbus is bus j, whose Yd thread j holds)
                if (__any_sync(__activemask(), j < nbus)) {
                    iv = fast_rcp(v);
                    if (j < nbus) {
                        const double tv = fix_twice(v), v2 = v * v;
                        sW2[j] = make_double2(__dmul_rn(tv, ydo.x), neg(__dmul_rn(tv, ydo.y)));   // 2 v conj(Yd)
                        sSv[j] = make_double2(__dmul_rn(v2, ydo.x), neg(__dmul_rn(v2, ydo.y)));   // v^2 conj(Yd)
                    }
                }
            } else if (j < nbus) {
                sW2[j].x = v * v;
            }
            sW[j] = make_double2(v, iv);
        }
        if (tid < nbus) {
            sbm[tid] = bmo;
            if (!JAC) syd[tid] = ydo;
            sord[tid] = ordo;
        }
        __syncthreads();
        PF_PROBE_MARK(1);

        // ---- evaluation: one terminal per thread ----
        for (int i = tid; i < nt; i += TB) {
            if (i != tid) {
                yf = a.tcfx[t0 + i];
                ey = a.tce[t0 + i];
                nq = a.tloc[t0 + i];
                ol = a.town[t0 + i];
            }
            ol -= b0;
            // G = conj(Yc) V_o conj(U_q) = dS_t/dv_q on the integer pipe (FP64
            // products for the values the fixed-point form does not hold)
            const longlong2 A = sA[ol], uq = sU[nq.x];
            const double vo = sW[ol].x, vq = sW[nq.x].x;
            double Gr, Gi;
            if (A.x == kFixNaN || uq.x == kFixNaN || ey == 0 ||
                !fix_G_fast(A.x, A.y, vo, uq.x, uq.y, yf.x, yf.y, ey, &Gr, &Gi)) {
                const longlong2 uo = sU[ol];
                const double2 yc = a.tcoup[t0 + i];
                fix_G(A.x, A.y, vo, uo.x, uo.y, uq.x, uq.y, 0, 0, 0, yc.x, yc.y, &Gr, &Gi);
            }
            const double Kr = vq * Gr, Ki = vq * Gi;   // K_t = v_q G
            if (JAC) {
                skg[2 * i] = make_double2(Kr, Ki);
                skg[2 * i + 1] = make_double2(Gr, Gi);
                skp[i] = nq.y;
                if (!(nq.y & EW_ACCUM)) {
                    const int4 bm = sbm[ol];
                    const int pos = bm.x + (nq.y & EW_KMASK), d = bm.y;
                    jst[pos] = Ki;           // J11 = Re(-j K)
                    jst[pos + d] = Gr;       // J12
                    jst[L + pos] = neg(Kr);  // J21 = Im(-j K)
                    jst[L + pos + d] = Gi;   // J22
                }
            } else {
                skg[i] = make_double2(Kr, Ki);
            }
        }
        __syncthreads();
        PF_PROBE_MARK(2);

        // ---- reduction: its terminals in sorted order onto every bus ----
        const int pqs = (int)sp.pqs, par = b0 & 1;
        if (JAC) {
            // two threads per bus: x = 2b' + im sums the real (im = 0) or imaginary
            // (im = 1) parts of K of bus b = sord[b'] and writes the entries that
            // depend on them only; the arithmetic is uniform across the pair (no
            // divergence), and with the buses taken by decreasing terminal count
            // the lanes of a warp loop about equally long
            const double *kg = reinterpret_cast<const double *>(skg);   // K.x, K.y, G.x, G.y per terminal
            for (int x = tid; x < 2 * nbus; x += TB) {
                const int b = sord[x >> 1], im = x & 1;
                const int4 bm = sbm[b];
                const int tend = b + 1 < nbus ? sbm[b + 1].w : nt;
                const int d = bm.y;
                // the sum starts from the first terminal (which starts its
                // parallel run, so it is never EW_ACCUM): one addition fewer
                int i = bm.w;
                double sK = 0.0;
                if (i < tend) sK = kg[4 * i++ + im];
                for (; i < tend; ++i) {
                    sK += kg[4 * i + im];
                    const int kp = skp[i];
                    if (kp & EW_ACCUM) {   // later branch of a parallel run: add into the run's slot
                        const int pos = bm.x + (kp & EW_KMASK);
                        if (im) {
                            jst[pos] += kg[4 * i + 1];           // J11 += Re(-j K)
                            jst[L + pos + d] += kg[4 * i + 3];   // J22 += Im G
                        } else {
                            jst[pos + d] += kg[4 * i + 2];       // J12 += Re G
                            jst[L + pos] -= kg[4 * i];           // J21 += Im(-j K)
                        }
                    }
                }
                const double2 dv = sW2[b], sv = sSv[b];   // 2 v conj(Yd), v^2 conj(Yd)
                const double iv = sW[b].y;
                const int pos = bm.x + bm.z;
                jst[(im ? 0 : L) + pos] = neg_if(sK, im);                  // Re / Im of j sum K
                jst[(im ? L : 0) + pos + d] = fma(sK, iv, im ? dv.y : dv.x);   // 2 v conj(Yd) + sum K / v
                spq[(im ? pqs : 0) + b + par] = sK + (im ? sv.y : sv.x);      // S = v^2 conj(Yd) + sum K
            }
        } else {
            // two threads per bus as above; v^2 from the phasor phase
            const double *k1 = reinterpret_cast<const double *>(skg);   // K.x, K.y per terminal
            for (int x = tid; x < 2 * nbus; x += TB) {
                const int b = sord[x >> 1], im = x & 1;
                const int4 bm = sbm[b];
                const int tend = b + 1 < nbus ? sbm[b + 1].w : nt;
                int i = bm.w;
                double sK = 0.0;
                if (i < tend) sK = k1[2 * i++ + im];
                for (; i < tend; ++i) sK += k1[2 * i + im];
                const double2 y = syd[b];
                const double v2 = sW2[b].x;
                spq[(im ? pqs : 0) + b + par] = fma(v2, im ? neg(y.y) : y.x, sK);   // S = v^2 conj(Yd) + sum K
            }
        }

        // ---- stores ----
        if (RED) {
            // J through a map from canonical positions (the reduced system's
            // CSC index, or a caller's pattern's position: Alg. 2's P_xy; -1
            // for an entry that is not kept), then the kept P and Q mismatches
            // to F, or P and Q themselves (no canonical J is written)
            __syncthreads();
            const long long p0 = 2 * (long long)r0, q0 = 2 * (long long)a.nnz + p0 - L;
            constexpr int U = 4;   // map loads in flight per thread and round (more spill at 48 registers)
            for (int base = tid; base < 2 * L; base += U * TB) {
                int k[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int x = base + u * TB;
                    k[u] = x < 2 * L ? a.jinv[(x < L ? p0 : q0) + x] : -1;
                }
#pragma unroll
                for (int u = 0; u < U; ++u)
                    if (k[u] >= 0) a.Jr[k[u]] = jst[base + u * TB];
            }
            if (a.binv)
                for (int b = tid; b < nbus; b += TB) {
                    const int2 e = a.binv[b0 + b];
                    if (e.x >= 0) a.F[e.x] = spq[b + par] - a.Ps[b0 + b];
                    if (e.y >= 0) a.F[e.y] = spq[pqs + b + par] - a.Qs[b0 + b];
                }
            if (a.P)
                for (int b = tid; b < nbus; b += TB) {
                    a.P[b0 + b] = spq[b + par];
                    a.Q[b0 + b] = spq[pqs + b + par];
                }
        } else if (a.aligned) {
            fence_proxy_async_smem();
            __syncthreads();
            PF_PROBE_MARK(3);
            if (tid == 0) {
                if (JAC) {
                    bulk_s2g(a.J + 2 * (long long)r0, jst, 8u * (uint32_t)L);
                    bulk_s2g(a.J + 2 * (long long)a.nnz + 2 * (long long)r0, jst + L, 8u * (uint32_t)L);
                }
                if (a.P) {
                    store_range(a.P, spq, b0, b1);
                    store_range(a.Q, spq + pqs, b0, b1);
                }
                bulk_commit();
                bulk_wait_read();   // shared memory stays allocated until the copies have read it
            }
        } else {
            __syncthreads();
            if (JAC) {
                double *Jp = a.J + 2 * (long long)r0;
                double *Jq = a.J + 2 * (long long)a.nnz + 2 * (long long)r0;
                for (int x = tid; x < L; x += TB) {
                    Jp[x] = jst[x];
                    Jq[x] = jst[L + x];
                }
            }
            if (a.P)
                for (int b = tid; b < nbus; b += TB) {
                    a.P[b0 + b] = spq[b + par];
                    a.Q[b0 + b] = spq[pqs + b + par];
                }
        }
#ifdef PF_PHASE_PROBE
        if (probe && tid == 0) {
            pt[4] = clock64() - pt0;
            unsigned int smid;
            asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
            unsigned long long *o = g_phase_probe + (long long)w * kProbeSlots;
            o[0] = gt0;
            o[1] = probe_gtimer();
            o[2] = smid;
            for (int k = 0; k < 5; ++k) o[3 + k] = (unsigned long long)pt[k];
            o[8] = gtw;
        }
#endif
        if (!PERSIST) break;
    }
}

// At most 48 registers: 5 CTAs of 256 or 10 of 128 threads per SM.
template <bool JAC>
__global__ void __launch_bounds__(256, 5) k_ew(EwArgs a)
{
    ew_windows<JAC, false>(a);
}

// the Jacobian evaluation with its outputs in host memory (persistent CTAs)
__global__ void __launch_bounds__(256, 5) k_ew_host(EwArgs a)
{
    ew_windows<true, true>(a);
}

// the Jacobian evaluation with its values stored through a position map: the
// reduced Newton system, or a caller's pattern (Alg. 2)
__global__ void __launch_bounds__(256, 5) k_ew_red(EwArgs a)
{
    ew_windows<true, false, true>(a);
}

static bool al16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

// persistent CTAs per SM of the host-output evaluation
constexpr int kEwHostCtasPerSm = 2;

enum class EwOut { device, host, reduced };

template <bool JAC>
static cudaError_t launch_ew(Grid *g, const double *vm, const double *va, double *P, double *Q, double *J,
                             cudaStream_t s, EwOut out, const double *Ps = nullptr, const double *Qs = nullptr,
                             double *F = nullptr, double *Jr = nullptr, const int *jinv = nullptr,
                             const int2 *binv = nullptr)
{
    const EwDev &L = g->ew;
    if (L.nwin == 0) return cudaSuccess;
    const int max_nph = L.max_nph;
    const EwSmem sp = ew_smem_plan(L.max_nbus, L.max_nt, JAC ? L.max_L : 0, JAC, max_nph);
    const uint32_t smem = sp.total + kTrigSmem;
    // outputs in host memory: persistent CTAs (kEwHostCtasPerSm per SM) loop
    // over the windows, so the host link carries the first windows' outputs
    // while the later ones are evaluated
    const bool persist = out == EwOut::host && JAC;
    const bool red = out == EwOut::reduced && JAC;
    uint32_t &conf = persist ? g->ew_smem_host : red ? g->ew_smem_red : JAC ? g->ew_smem_jac : g->ew_smem_inj;
    // conf: the largest size this grid has ensured (the process-wide limit
    // only grows, so a size ensured once stays valid)
    if (smem > 48u * 1024u && smem > conf) {
        cudaError_t e = ensure_dyn_smem(
            reinterpret_cast<const void *>(persist ? k_ew_host : red ? k_ew_red : k_ew<JAC>), smem);
        if (e != cudaSuccess) return e;
        conf = smem;
    }
    int grid = L.nwin;
    if (persist) {
        if (g->nsm == 0) {
            int dev = 0;
            cudaError_t e = cudaGetDevice(&dev);
            if (e == cudaSuccess) e = cudaDeviceGetAttribute(&g->nsm, cudaDevAttrMultiProcessorCount, dev);
            if (e != cudaSuccess) return e;
        }
        grid = std::min(grid, kEwHostCtasPerSm * g->nsm);
    }
    EwArgs a = {};
    a.nnz = g->nnz;
    a.nwin = L.nwin;
    a.max_nbus = L.max_nbus;
    a.max_nt = L.max_nt;
    a.max_L = L.max_L;
    a.max_nph = max_nph;
    // bulk (TMA) stores for device outputs; plain coalesced stores for host memory
    a.aligned = out == EwOut::device && (!J || al16(J)) && (!P || (al16(P) && al16(Q)));
    a.desc = L.desc;
    a.slotbus = L.slotbus;
    a.bmeta = L.bmeta;
    a.rorder = L.rorder;
    a.town = g->town;
    a.yd = g->bus_yd;
    a.tcoup = g->tcoup;
    a.tcfx = g->tcfx;
    a.tce = g->tce;
    a.trig = trig_table();
    a.tloc = L.tloc;
    a.vm = vm;
    a.va = va;
    a.P = P;
    a.Q = Q;
    a.J = J;
    if (red) {
        a.jinv = jinv;
        a.binv = binv;
        a.Ps = Ps;
        a.Qs = Qs;
        a.F = F;
        a.Jr = Jr;
    }
    // the device-output kernels are launched as programmatic dependents of
    // the previous kernel in the stream (their prologue overlaps its end)
    if (persist) {
        k_ew_host<<<(unsigned)grid, (unsigned)L.tb, smem, s>>>(a);
        return cudaGetLastError();
    }
    if (red) return launch_k(k_ew_red, grid, L.tb, smem, s, true, a);
    return launch_k(k_ew<JAC>, grid, L.tb, smem, s, true, a);
}

cudaError_t ew_blocks_per_sm(int tb, size_t smem, int *per_sm)
{
    if (smem > 48u * 1024u) {
        cudaError_t e = ensure_dyn_smem(reinterpret_cast<const void *>(k_ew<true>), smem);
        if (e != cudaSuccess) return e;
    }
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_ew<true>, tb, smem);
}

cudaError_t launch_jac_ew(Grid *g, const double *vm, const double *va, double *P, double *Q, double *J,
                          cudaStream_t s, bool host_out)
{
    return launch_ew<true>(g, vm, va, P, Q, J, s, host_out ? EwOut::host : EwOut::device);
}

cudaError_t launch_jac_ew_reduced(Grid *g, const double *vm, const double *va, const double *Ps, const double *Qs,
                                  double *F, double *Jr, cudaStream_t s)
{
    return launch_ew<true>(g, vm, va, nullptr, nullptr, nullptr, s, EwOut::reduced, Ps, Qs, F, Jr, g->red_jinv,
                           g->red_binv);
}

cudaError_t launch_jac_ew_mapped(Grid *g, const double *vm, const double *va, double *P, double *Q, const int *map,
                                 double *Jt, cudaStream_t s)
{
    return launch_ew<true>(g, vm, va, P, Q, nullptr, s, EwOut::reduced, nullptr, nullptr, nullptr, Jt, map,
                           nullptr);
}

cudaError_t launch_inj_ew(Grid *g, const double *vm, const double *va, double *P, double *Q, cudaStream_t s)
{
    return launch_ew<false>(g, vm, va, P, Q, nullptr, s, EwOut::device);
}

}  // namespace pf

PF_API pf_status pf_phase_probe_read(uint64_t *out, int32_t max_windows, int32_t *nwin)
{
#ifdef PF_PHASE_PROBE
    using namespace pf;
    if (!out || max_windows < 0) return set_error(PF_EINVAL, "pf_phase_probe_read: NULL output or negative size");
    const int n = max_windows < kProbeMaxWin ? max_windows : kProbeMaxWin;
    if (n > 0)
        PF_CUDA(cudaMemcpyFromSymbol(out, g_phase_probe, (size_t)n * kProbeSlots * sizeof(unsigned long long)));
    if (nwin) *nwin = n;
    return PF_OK;
#else
    (void)out;
    (void)max_windows;
    if (nwin) *nwin = 0;
    return pf::set_error(PF_EUNSUPPORTED, "pf_phase_probe_read: library built without -DPF_PHASE_PROBE");
#endif
}
