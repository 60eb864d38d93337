// pd_stencil2d_walk.cu -- FP32 2D stiffness product K u (the bond sum of
// Eq. mat:f1, i.e. the TBT form of Sec. 3.2-3.4) as a column walk, for sm_103a.
//
// A CTA owns a strip of 128 grid columns (four warps side by side, one column
// per lane) and walks down it.  Rows arrive in shared memory as TMA boxes of
// 2M+1 rows (both components, 4 halo columns on each side, zero fill outside
// the grid) into a ring of four slots; the warp that releases a slot last
// refills it, so no warp waits for another unless it runs a whole ring ahead.
//
// The sum is taken as differences of nearby values (its FP32 error stays
// relative to |K u| on smooth fields too).  With H_ox(i) = u(x+ox, i) - u(x, i),
// V_k(j) = u(x, j+k) - u(x, j) and, per column offset ox,
//   E(i) = H_ox(i) + H_-ox(i)   (horizontal second difference of row i),
//   G(i) = u(x+ox, i) - u(x-ox, i),
// the output at row r is
//   (K u)(r) = sum_ox [ cxx(ox,0) E_x(r) + sum_k c1(ox,k) (E(r+k) + E(r-k))
//                                         + c2(ox,k) (G(r+k) - G(r-k)) ]
//              + sum_k Cbar(k) (V_k(r) - V_k(r-k)),
// c1 = (cxx, cyy), c2 = (cxy, cxy) (a2 swapped at the end), Cbar(k) the sum of
// the diagonal blocks over the offsets with |oy| = k.  Instead of gathering
// these per output, every loaded row is formed once (E, G per ox, V_k for the
// M rows above it) and scattered into the accumulators of the 2M+1 outputs it
// touches; an output is complete, and stored, once the row M below it has been
// scattered.  The accumulators sit in registers indexed by the row modulo 2M+1
// (the box height), so every index is a compile-time constant.
//
// Per output at M = 3: 12 shared loads, about 35 FP32x2 and 8 FP32 operations
// (the 64 x 32 tile kernel of pd_stencil2d_tma.cu: 17.7 loads and about 97
// instructions), and no vertical halo: every input row is staged once per
// strip.  Every output runs the same operation sequence wherever its
// strip segment begins, so a band of rows (pd_matvec_rows) reproduces the
// whole-grid product bit for bit.
//
// Boundaries: for lanes whose horizon leaves the grid on the left or right
// (edge strips) each H is multiplied by the lane's in-grid flag of that
// column, and the vertical term takes per-lane coefficients (see lane_coefs);
// for boxes that touch the top or bottom of the grid each V_k(j) is dropped
// unless rows j and j+k both lie in the grid.  Rows outside the grid are zero
// in the box, so their E and G vanish by themselves.  The result is the
// in-grid bond sum of Eq. mat:f1 (no diagonal table, no cancelling D^e term).
//
// Used for FP32 2D products with M <= 3 (beyond, the register windows spill) and a row length that is a multiple of
// 4 floats (TMA stride rule), without projection or a fused dot; the tile
// kernel serves the rest.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstring>

#include "pd_stencil.cuh"
#include "pd_tma2d.cuh"

namespace pd {

namespace {

using namespace tma2d;

constexpr int kWW = 32;                // columns per warp (one per lane)
constexpr int kWarps = 4;              // warps per CTA, side by side
constexpr int kSW = kWW * kWarps;      // columns per CTA strip (128)
constexpr int kWXL = 4;                // halo columns staged on each side (M <= 3 used)
constexpr int kWBX = kSW + 2 * kWXL;   // staged row length: 136 floats = 544 bytes
constexpr int kSlots = 4;              // ring slots per CTA (three boxes in flight)
constexpr int kRep = 1;                // accumulator periods (2M+1 rows) per box

template <int M>
__host__ __device__ constexpr int wtb() { return 2 * M + 1; }   // accumulator period (rows)
template <int M>
__host__ __device__ constexpr int wbox() { return kRep * wtb<M>(); }   // rows per box
template <int M>
__host__ __device__ constexpr int wslot_bytes() { return (2 * wbox<M>() * kWBX * 4 + 127) / 128 * 128; }
template <int M>
__host__ __device__ constexpr int kmax_of(int ox) { return isqrt_c(M * M - ox * ox); }
// number of (ox, k) pairs with 1 <= ox < M, 1 <= k <= kmax(ox); index of one
template <int M>
__host__ __device__ constexpr int n_pairs_walk()
{
    int n = 0;
    for (int ox = 1; ox < M; ++ox) n += kmax_of<M>(ox);
    return n;
}
template <int M>
__host__ __device__ constexpr int pidx(int ox, int k)
{
    int n = 0;
    for (int x = 1; x < ox; ++x) n += kmax_of<M>(x);
    return n + k - 1;
}

// Coefficients premultiplied by -scale (so that K u = a1 + swap(a2)).
template <int M>
struct __align__(16) WalkTab {
    static constexpr int kNP = n_pairs_walk<M>() > 0 ? n_pairs_walk<M>() : 1;
    u64 c1[kNP], c2[kNP];             // (cxx, cyy), (cxy, cxy) of (ox, k)
    u64 cb[M];                        // Cbar(k)
    u64 cv0[M];                       // (0, cyy(0, k)): the axis pair (0, k) alone (edge lanes)
    float cax[M];                     // cxx(ox, 0)
};

// Edge lanes: in-grid flags of the columns x +- ox and the per-lane vertical
// coefficients.  For a pair (ox, +-k) whose ends may leave the grid, the
// vertical parts V of the two ends combine to
//   (m+ + m-) diag(c) (V_k(r) - V_k(r-k)) + (m+ - m-) cxy (V_k(r) + V_k(r-k))
// (m+- the flags of x +- ox); summed over ox with the axis pair (0, k) this
// gives cb(k) for a1 and d(k) for a2.
template <int M>
struct LaneCoefs {
    u64 mp[M], mm[M];      // (m, m) flags of x + ox, x - ox
    u64 cb[M], d[M];
};

template <int M>
__device__ __forceinline__ void lane_coefs(const WalkTab<M> &tab, int x, int nx, LaneCoefs<M> &lc)
{
#pragma unroll
    for (int ox = 1; ox <= M; ++ox) {
        const float p = (x + ox < nx) ? 1.f : 0.f, m = (x - ox >= 0) ? 1.f : 0.f;
        lc.mp[ox - 1] = pk(p, p);
        lc.mm[ox - 1] = pk(m, m);
    }
#pragma unroll
    for (int k = 1; k <= M; ++k) {
        float2 cb = upk(tab.cv0[k - 1]), d = make_float2(0.f, 0.f);
        static_for<1, M>([&](auto OX) {
            constexpr int ox = decltype(OX)::value;
            if (k <= kmax_of<M>(ox)) {
                const float2 c1 = upk(tab.c1[pidx<M>(ox, k)]), c2 = upk(tab.c2[pidx<M>(ox, k)]);
                const float s = upk(lc.mp[ox - 1]).x + upk(lc.mm[ox - 1]).x;
                const float t = upk(lc.mp[ox - 1]).x - upk(lc.mm[ox - 1]).x;
                cb.x = __fmaf_rn(s, c1.x, cb.x);
                cb.y = __fmaf_rn(s, c1.y, cb.y);
                d.x = __fmaf_rn(t, c2.x, d.x);
            }
        });
        d.y = d.x;
        lc.cb[k - 1] = pk(cb.x, cb.y);
        lc.d[k - 1] = pk(d.x, d.y);
    }
}

// Register windows carried from box to box: the own column of the last M rows,
// V_k of the last k rows, and G of each column offset over its last 2 kmax rows.
template <int M>
struct WalkWin {
    static constexpr int kNG = 2 * (kmax_of<M>(1) > 0 ? kmax_of<M>(1) : 1);
    u64 w[wtb<M>()];                 // u(x, row), indexed by row mod P
    u64 v[M][wtb<M>()];              // V_k(j) = u(x, j + k) - u(x, j), indexed by (j + k) mod P
    u64 g[M > 1 ? M - 1 : 1][wtb<M>()];   // G_ox(row), indexed by row mod P
};

// One box: rows q = 0..P-1 of the slot (grid rows row0 + q), scattered into the
// accumulators; the output of slot q is complete after row q and is stored when
// valid.  Every difference that the sum needs is formed before it is
// multiplied, so that terms of the size of first differences never cancel in
// an accumulator:
//   a1(r) += c1 E(r +- k)              at rows r -+ k,
//   a2(r) += c2 (G(r + k) - G(r - k))   at row r + k,
//   a1(r) += Cbar(k) (V_k(r) - V_k(r - k))   at row r + k.
//   XE: edge strip (per-lane flags); YE: the box touches the top or bottom rows.
// rho0: segment-relative index of row 0; outputs rho in [2M, lim) are stored.
//   ALLV: every output of the box is stored (no per-row tests).
// o0: the output of row 0 of the box (x component; y at o0 + comp_stride).
template <int M, bool XE, bool YE, bool ALLV>
__device__ __forceinline__ void walk_box(const float *__restrict__ rx0, const WalkTab<M> &tab, const LaneCoefs<M> &lc,
                                         u64 (&a1)[wtb<M>()], u64 (&a2)[wtb<M>()], WalkWin<M> &wn,
                                         int row0, int ny, int rho0, int lim, bool lane_ok,
                                         float *__restrict__ o0, int row_stride, int64_t comp_stride)
{
    constexpr int P = wtb<M>();
    constexpr int KD = kmax_of<M>(1);   // farthest row below that a loaded row touches
    static_for<0, P>([&](auto Q) {
        constexpr int q = decltype(Q)::value;
        const float *rx = rx0 + q * kWBX, *ry = rx + wbox<M>() * kWBX;   // x and y planes of the box
        const u64 w = pk(rx[0], ry[0]);
        // vertical: V_k(j) for j = row - k, then W_k and (edge lanes) the central sum of output j
        static_for<1, M + 1>([&](auto K) {
            constexpr int k = decltype(K)::value;
            u64 V = fsub2(w, wn.w[(q - k + P) % P]);
            if constexpr (YE) {
                const int i = row0 + q;
                if (!(i < ny && i - k >= 0)) V = 0ull;
            }
            const u64 Vold = wn.v[k - 1][(q - k + P) % P];   // V_k(j - k)
            wn.v[k - 1][q] = V;
            constexpr int sl = ((q - k + M) % P + P) % P;    // output j = row - k
            if constexpr (XE) {
                a1[sl] = ffma2(lc.cb[k - 1], fsub2(V, Vold), a1[sl]);
                if constexpr (k == 1)
                    a2[sl] = fmul2(lc.d[k - 1], fadd2(V, Vold));
                else
                    a2[sl] = ffma2(lc.d[k - 1], fadd2(V, Vold), a2[sl]);
            } else {
                a1[sl] = ffma2(tab.cb[k - 1], fsub2(V, Vold), a1[sl]);
            }
        });
        wn.w[q] = w;
        // column offsets with pairs (ox, +-k): E scattered to rows q -+ k, G differenced with 2k rows above
        static_for<1, M>([&](auto OX) {
            constexpr int ox = decltype(OX)::value;
            const u64 wp = pk(rx[ox], ry[ox]), wm = pk(rx[-ox], ry[-ox]);
            u64 E, G;
            if constexpr (XE) {
                const u64 hp = fmul2(lc.mp[ox - 1], fsub2(wp, w)), hm = fmul2(lc.mm[ox - 1], fsub2(wm, w));
                E = fadd2(hp, hm);
                G = fsub2(hp, hm);
            } else {
                E = fadd2(fsub2(wp, w), fsub2(wm, w));
                G = fsub2(wp, wm);
            }
            {   // axis pair (ox, 0): x component only
                constexpr int s0 = (q + M) % P;
                float2 acc = upk(a1[s0]);
                acc.x = __fmaf_rn(tab.cax[ox - 1], upk(E).x, acc.x);
                a1[s0] = pk(acc.x, acc.y);
            }
            static_for<1, kmax_of<M>(ox) + 1>([&](auto K) {
                constexpr int k = decltype(K)::value;
                constexpr int pi = pidx<M>(ox, k);
                constexpr int sp = (q + k + M) % P, sm = ((q - k + M) % P + P) % P;
                if constexpr (ox == 1 && k == KD)   // first contribution to the output k rows down
                    a1[sp] = fmul2(tab.c1[pi], E);
                else
                    a1[sp] = ffma2(tab.c1[pi], E, a1[sp]);
                a1[sm] = ffma2(tab.c1[pi], E, a1[sm]);
                const u64 dG = fsub2(G, wn.g[ox - 1][(q - 2 * k + 2 * P) % P]);   // G(r + k) - G(r - k), r = row - k
                if constexpr (!XE && ox == 1 && k == 1)
                    a2[sm] = fmul2(tab.c2[pi], dG);
                else
                    a2[sm] = ffma2(tab.c2[pi], dG, a2[sm]);
            });
            wn.g[ox - 1][q] = G;
        });
        {   // outermost column offset (M, 0): x component only
            const float wx = upk(w).x;
            float e;
            if constexpr (XE)
                e = __fmaf_rn(upk(lc.mp[M - 1]).x, rx[M] - wx, upk(lc.mm[M - 1]).x * (rx[-M] - wx));
            else
                e = (rx[M] - wx) + (rx[-M] - wx);
            constexpr int s0 = (q + M) % P;
            float2 acc = upk(a1[s0]);
            acc.x = __fmaf_rn(tab.cax[M - 1], e, acc.x);
            a1[s0] = pk(acc.x, acc.y);
        }
        // the output of slot q (the row M above) is complete
        {
            const float2 x1 = upk(a1[q]), x2 = upk(a2[q]);
            if (ALLV || (lane_ok && rho0 + q >= 2 * M && rho0 + q < lim)) {
                float *o = o0 + q * row_stride;
                o[0] = x1.x + x2.y;
                o[comp_stride] = x1.y + x2.x;
            }
            if constexpr (KD == 0) {   // M = 1: no pair writes a first contribution
                a1[q] = 0ull;
                if constexpr (!XE) a2[q] = 0ull;
            }
        }
    });
}

// Bounded wait on a box, giving up early once another warp of the CTA has given up.
__device__ __forceinline__ bool box_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag)
{
    for (int it = 0; it < (1 << 22); ++it) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
        if (ok) return true;
        if ((it & 255) == 255 && *abort_flag) return false;
    }
    return false;
}

// One release of a ring slot by a warp (acquire-release at CTA scope); returns
// the number of releases before it.
__device__ __forceinline__ uint32_t slot_release(uint32_t *cnt)
{
    uint32_t old;
    asm volatile("atom.acq_rel.cta.shared::cta.add.u32 %0, [%1], 1;" : "=r"(old) : "r"(smem_u32(cnt)) : "memory");
    return old;
}

// The CTA owns a strip of 128 columns (four warps side by side) and walks down
// its share of the (strip, row) positions of the batch; every box is one TMA
// copy of 136 x (2M+1) x 2 floats shared by the four warps.  The warp that
// releases a slot last refills it, so no warp waits for another unless it runs
// a whole ring ahead.
template <int M>
__global__ void __launch_bounds__(kWarps * 32, 4)
k_tbt2d_walk(const __grid_constant__ CUtensorMap map, float *__restrict__ out, int nx, int ny, int64_t Nout,
             int in_row0, int out_row0, int out_rows, int nstrips, int64_t total, WalkTab<M> tab, int *err)
{
    constexpr int P = wtb<M>(), TB = wbox<M>();
    constexpr uint32_t kBytes = 2u * TB * kWBX * sizeof(float);
    constexpr int SLOT = wslot_bytes<M>() / 4;   // floats per slot
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t full[kSlots];
    __shared__ uint32_t cnt[kSlots];
    __shared__ int last_box[kSlots];
    __shared__ int s_abort;
    float *const ring = reinterpret_cast<float *>(smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int k = 0; k < kSlots; ++k) {
            mbar_init(&full[k], 1);
            cnt[k] = 0;
            last_box[k] = -1;
        }
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    // The CTA's share of the positions (strip c, output row) in c-major order.
    const int64_t nB = gridDim.x, bid = blockIdx.x;
    const int64_t begin = total * bid / nB, end = total * (bid + 1) / nB;
    const int H = out_rows;
    struct Seg {
        int64_t c;
        int a, e, nb;
    };
    auto seg_at = [&](int64_t pos, Seg &s) -> bool {
        if (pos >= end) return false;
        s.c = (pos >> 31) ? pos / H : (int64_t)((uint32_t)pos / (uint32_t)H);   // 32-bit division when it fits
        s.a = (int)(pos - s.c * H);
        s.e = (int)min((int64_t)H, end - s.c * H);
        s.nb = (s.e - s.a + 2 * M + TB - 1) / TB;
        return true;
    };
    // the box list, kSlots boxes ahead of consumption (every thread keeps its own copy)
    Seg ps;
    bool pv = seg_at(begin, ps);
    int pbox = 0;
    auto advance_producer = [&]() {
        if (++pbox == ps.nb) {
            pv = seg_at(ps.c * H + ps.e, ps);
            pbox = 0;
        }
    };
    auto issue = [&](uint32_t k) {   // box k of the list, at the producer's position
        const int b = (int)ps.c / nstrips, strip = (int)ps.c - b * nstrips;
        const int row = out_row0 + ps.a - M + pbox * TB - in_row0;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_tx(&full[k % kSlots], kBytes);
        tma_load_3d(ring + (k % kSlots) * SLOT, &map, strip * kSW - kWXL, row, 2 * b, &full[k % kSlots]);
        last_box[k % kSlots] = (int)k;
    };
    for (uint32_t k = 0; k < (uint32_t)kSlots && pv; ++k) {
        if (threadIdx.x == 0) issue(k);
        advance_producer();
    }

    Seg cs;
    bool cv = seg_at(begin, cs);
    uint32_t kc = 0;
    bool aborted = false;
    u64 a1[P], a2[P];
    WalkWin<M> wn;
    auto segment = [&](auto XEV) {
        constexpr bool XE = decltype(XEV)::value;
        const int b = (int)cs.c / nstrips, strip = (int)cs.c - b * nstrips;
        const int x = strip * kSW + warp * kWW + lane;
        const bool lane_ok = x < nx;
        const bool warp_full = strip * kSW + warp * kWW + kWW <= nx;
        LaneCoefs<M> lc;
        if constexpr (XE) lane_coefs<M>(tab, x, nx, lc);
        const int row_base = out_row0 + cs.a - M;   // grid row of the segment's first loaded row
        // the output of segment-relative row rho is grid row out_row0 + a - 2M + rho
        float *const optr = out + (int64_t)b * 2 * Nout + (int64_t)(cs.a - 2 * M) * nx + x;
        const int lim = cs.e - cs.a + 2 * M;
#pragma unroll
        for (int i = 0; i < P; ++i) {
            a1[i] = a2[i] = wn.w[i] = 0ull;
#pragma unroll
            for (int k = 0; k < M; ++k) wn.v[k][i] = 0ull;
#pragma unroll
            for (int k = 0; k < (M > 1 ? M - 1 : 1); ++k) wn.g[k][i] = 0ull;
        }
        for (int cbox = 0; cbox < cs.nb; ++cbox) {
            const uint32_t slot = kc % kSlots;
            const bool ok = box_wait(&full[slot], (kc / kSlots) & 1, &s_abort);
            if (__any_sync(0xffffffffu, !ok)) {   // warp-uniform
                if (lane == 0) {
                    atomicExch(err, 1);
                    s_abort = 1;
                }
                aborted = true;
                return;
            }
            const float *rxb = ring + slot * SLOT + kWXL + warp * kWW + lane;
            static_for<0, kRep>([&](auto R) {
                constexpr int rep = decltype(R)::value;
                const float *rx0 = rxb + rep * P * kWBX;
                const int rho0 = cbox * TB + rep * P;
                const int row0 = row_base + rho0;
                float *const o0 = optr + (int64_t)rho0 * nx;
                const bool ye = row0 - M < 0 || row0 + P > ny;
                const bool allv = warp_full && rho0 >= 2 * M && rho0 + P <= lim;
                if (ye) {
                    walk_box<M, XE, true, false>(rx0, tab, lc, a1, a2, wn, row0, ny, rho0, lim, lane_ok, o0, nx, Nout);
                } else if (allv) {
                    walk_box<M, XE, false, true>(rx0, tab, lc, a1, a2, wn, row0, ny, rho0, lim, lane_ok, o0, nx, Nout);
                } else {
                    walk_box<M, XE, false, false>(rx0, tab, lc, a1, a2, wn, row0, ny, rho0, lim, lane_ok, o0, nx, Nout);
                }
            });
            // this warp's reads of the slot are done; the last of the four refills it
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            uint32_t old = 0;
            if (lane == 0) old = slot_release(&cnt[slot]);
            old = __shfl_sync(0xffffffffu, old, 0);
            if (old == (kc / kSlots) * kWarps + (kWarps - 1) && pv && lane == 0) issue(kc + kSlots);
            if (pv) advance_producer();
            ++kc;
        }
    };
    while (cv && !aborted) {
        const int strip = (int)cs.c % nstrips, x0 = strip * kSW + warp * kWW;
        if (x0 < M || x0 + kWW > nx - M)
            segment(std::true_type{});
        else
            segment(std::false_type{});
        cv = seg_at(cs.c * H + cs.e, cs);
    }
    __syncthreads();
    if (s_abort && threadIdx.x == 0)   // let the copies still in flight land before the CTA exits
        for (int k = 0; k < kSlots; ++k)
            if (last_box[k] >= 0) mbar_wait(&full[k], ((uint32_t)last_box[k] / kSlots) & 1);
}

// Tensor map over `batch` fields of two FP32 planes [2*batch][rows][nx] with a
// box of box_w x box_h x 2; false if the driver rejects it.
bool make_map_box(CUtensorMap *map, const void *base, int nx, int rows, int64_t batch, int box_w, int box_h)
{
    EncodeTiledFn enc = encode_fn();
    if (!enc) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)rows, (cuuint64_t)(2 * batch)};
    const cuuint64_t strides[2] = {(cuuint64_t)nx * sizeof(float), (cuuint64_t)nx * rows * sizeof(float)};
    const cuuint32_t box[3] = {(cuuint32_t)box_w, (cuuint32_t)box_h, 2};
    const cuuint32_t estr[3] = {1, 1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void *>(base), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int M>
WalkTab<M> make_walk(const pd_grid *g, double scale)
{
    WalkTab<M> t{};
    double c[6];
    double cb[M + 1][2] = {};
    auto p2 = [](double a, double b) {
        const float fa = (float)a, fb = (float)b;
        u64 r;
        uint32_t ua, ub;
        memcpy(&ua, &fa, 4);
        memcpy(&ub, &fb, 4);
        r = (u64)ua | ((u64)ub << 32);
        return r;
    };
    for (int ox = 1; ox <= M; ++ox) {
        coef_of(g, ox, 0, 0, false, c);   // xx, xy, yy
        t.cax[ox - 1] = (float)(-scale * c[0]);
        for (int k = 1; k <= kmax_of<M>(ox); ++k) {
            coef_of(g, ox, k, 0, false, c);
            if (ox < M) {
                const int pi = pidx<M>(ox, k);
                t.c1[pi] = p2(-scale * c[0], -scale * c[2]);
                t.c2[pi] = p2(-scale * c[1], -scale * c[1]);
            }
            cb[k][0] += 2 * c[0];
            cb[k][1] += 2 * c[2];
        }
    }
    for (int k = 1; k <= M; ++k) {
        coef_of(g, 0, k, 0, false, c);
        cb[k][1] += c[2];
        t.cv0[k - 1] = p2(0.0, -scale * c[2]);
        t.cb[k - 1] = p2(-scale * cb[k][0], -scale * cb[k][1]);
    }
    return t;
}

template <int M>
int run(pd_grid *g, const MatvecArgs &a, cudaStream_t s)
{
    constexpr int P = wtb<M>();
    const int nx = (int)g->n[0], ny = (int)g->n[1];
    const int in_row0 = (int)a.in_row0, in_rows = a.in_rows < 0 ? ny : (int)a.in_rows;
    const int out_row0 = (int)a.out_row0, out_rows = a.out_rows < 0 ? ny : (int)a.out_rows;
    CUtensorMap map;
    if (!make_map_box(&map, a.u, nx, in_rows, a.batch, kWBX, wbox<M>())) return fail(PD_ERR_CUDA, "tensor map encode failed");
    const size_t smem = (size_t)kSlots * wslot_bytes<M>();
    auto kern = k_tbt2d_walk<M>;
    static int attr_done[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && !attr_done[dev]) {
        PD_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        attr_done[dev] = 1;
    }
    const int nstrips = (nx + kSW - 1) / kSW;
    const int64_t total = (int64_t)a.batch * nstrips * out_rows;
    int occ = 0, sms = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kWarps * 32, smem);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (occ < 1) occ = 1;
    // at least ~48 rows per CTA, so that the 2M-row start of each segment stays small
    const int64_t want = (total + 47) / 48;
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)occ * sms));
    kern<<<blocks, kWarps * 32, smem, s>>>(map, (float *)a.out, nx, ny, (int64_t)out_rows * nx, in_row0, out_row0,
                                           out_rows, nstrips, total, make_walk<M>(g, a.scale), g->d_err);
    PD_CUDA(cudaGetLastError());
    return PD_OK;
}

}  // namespace

bool walk_stencil_eligible(const pd_grid *g, const MatvecArgs &a)
{
    return g->dim == 2 && g->M >= 1 && g->M <= 3 && !a.project && !a.dot_partial && !a.pair_form &&
           g->n[1] >= 1;
}

int run_tbt2d_walk(pd_grid *g, const MatvecArgs &a, cudaStream_t s)
{
    switch (g->M) {
        case 1: return run<1>(g, a, s);
        case 2: return run<2>(g, a, s);
        case 3: return run<3>(g, a, s);
    }
    return fail(PD_ERR_INVALID, "horizon M not compiled for the column walk");
}

}  // namespace pd
