// pic_particle_kernel.cuh -- the particle side of the PIC cycle on sm_103a,
// templated on the arithmetic of the particle push (included by one
// translation unit per precision and dimensionality:
// pic_particles_{f64,dd,f32}_{3d,2d}.cu).
//
// pic_particle_kernel: persistent CTAs pull work units (a chunk of one box's
// particles) from cost-ordered lists.  For every tile (sub-box) a unit touches,
// the guard-extended E/B tile is staged into shared memory by TMA
// (cp.async.bulk.tensor, local HBM only, no multicast).  The current goes
// straight into the guard-padded global J arrays as fire-and-forget FP64
// reductions (red.global.add.f64, performed in L2) in every precision; the
// FP32 variant also stages its particle loads through shared memory with
// cp.async one loop iteration ahead.  Each thread brackets its particle
// loop with clock64(); the deltas are warp-reduced, summed in shared memory and
// added once per unit to the box's cost -- the device-clock cost of
// arXiv 2104.11385 Sec. 2.2 (Fig. 2a); thread 0 adds the unit's %globaltimer
// span to the box's kernel-time cost.  The same pass writes each particle's new
// tile key and the per-tile histogram for the re-sort.
//
// Physics per particle (the schemes the paper leaves open, Sec. 2.1): field
// gather with B-spline shapes of order 1-3 at each component's Yee location
// (same order in every direction, or the energy-conserving variant with one
// order less along the staggered directions), relativistic Boris push,
// Esirkepov charge-conserving deposit (Esirkepov 2001).  The cost capture can
// be switched off per simulation to measure its overhead.
#pragma once
#include <type_traits>

#include "pic_dd.cuh"
#include "pic_internal.h"
#include "pic_sync.cuh"

namespace {

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z,
                                            uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Exact floor and fractional part of x.  On GB300 every FP64 instruction,
// conversions included, issues at the FP64 rate (about 2 per SM per clock), so
// for 0 <= x < 2^31 both come from integer work on the IEEE-754 bits; other x
// go through floor().  Both routes give the identical (exact) results.  The
// floor() route is a separate function: inlined, the compiler predicates it,
// and its FP64 instructions then occupy the FP64 pipe on every call.
struct IFrac {
    int i;
    double f;
};
static __device__ __noinline__ IFrac ifloor_frac_slow(double x) {
    const double fl = floor(x);
    return IFrac{(int)fl, x - fl};
}
static __device__ __noinline__ int ifloor_slow(double x) { return (int)floor(x); }

__device__ __forceinline__ int ifloor_frac(double x, double& f) {
    const long long b = __double_as_longlong(x);
    const int e = (int)((unsigned long long)b >> 52) - 1023;  // sign set -> e > 1023
    if (e < 0) {
        if (b >= 0) {  // 0 <= x < 1
            f = x;
            return 0;
        }
    } else if (e < 31) {
        const unsigned long long m = ((unsigned long long)b & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull;
        const int sh = 52 - e;
        const int i = (int)(m >> sh);
        const unsigned long long fm = m & ((1ull << sh) - 1ull);
        if (fm == 0ull) {
            f = 0.0;
        } else {
            const int top = 63 - __clzll((long long)fm);
            const unsigned long long bits = ((unsigned long long)(top - sh + 1023) << 52) |
                                            ((fm << (52 - top)) & 0xFFFFFFFFFFFFFull);
            f = __longlong_as_double((long long)bits);
        }
        return i;
    }
    const IFrac r = ifloor_frac_slow(x);
    f = r.f;
    return r.i;
}

// floor of x >= 0 (x < 2^31) by integer work; floor() otherwise
__device__ __forceinline__ int ifloor(double x) {
    const long long b = __double_as_longlong(x);
    const int e = (int)((unsigned long long)b >> 52) - 1023;
    if (e < 0 && b >= 0) return 0;
    if (e >= 0 && e < 31)
        return (int)((((unsigned long long)b & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull) >> (52 - e));
    return ifloor_slow(x);
}

// periodic image of a position that left [0, n) by less than n: a separate
// function, so that the rare FP64 add is a branch and not a predicated
// instruction holding the FP64 pipe for every particle
static __device__ __noinline__ double wrap_periodic(double x, double n) { return x < 0.0 ? x + n : x - n; }

// x < 0 and x >= y for y > 0 by integer comparison of the bit patterns
__device__ __forceinline__ bool is_neg(double x) { return __double_as_longlong(x) < 0; }
__device__ __forceinline__ bool ge_pos(double x, double y) {
    return __double_as_longlong(x) >= __double_as_longlong(y);
}
__device__ __forceinline__ bool ge_half(double f) {  // f >= 0.5 for f >= 0
    return __double_as_longlong(f) >= 0x3FE0000000000000ll;
}

// one-dimensional B-spline support: first node and ORDER+1 weights in the
// arithmetic type R (double; dd for the float-float variant; float for the FP32 one)
template <int ORDER, class R>
struct Support {
    int s;
    R w[ORDER + 1];
};

// cubic B-spline weights of the four nodes floor(xi)-1 .. floor(xi)+2, f = frac(xi)
template <class R>
__device__ __forceinline__ void cubic_weights(R f, R* w) {
    using A = Arith<R>;
    const R k6 = A::c(1.0 / 6.0), k23 = A::c(2.0 / 3.0), half = A::c(0.5);
    const R g = A::c(1.0) - f;
    const R f2 = f * f, g2 = g * g;
    w[0] = (g2 * g) * k6;
    w[1] = fma(half * f, f2, k23 - f2);
    w[2] = fma(half * g, g2, k23 - g2);
    w[3] = (f2 * f) * k6;
}

// support of a node-centred quantity at xi (cells, from the tile origin)
template <int ORDER, class R>
__device__ __forceinline__ Support<ORDER, R> support(double xi) {
    using A = Arith<R>;
    Support<ORDER, R> r;
    double f;
    const int i = ifloor_frac(xi, f);
    if constexpr (ORDER == 1) {
        r.s = i;
        const R fr = A::from(f);
        r.w[0] = A::c(1.0) - fr;
        r.w[1] = fr;
    } else if constexpr (ORDER == 2) {
        // nearest node c = floor(xi + 1/2), d = xi - c in [-1/2, 1/2)
        const bool up = ge_half(f);
        const R fr = A::from(f);
        const R d = up ? fr - A::c(1.0) : fr;
        const R a = A::c(0.5) - d, b = A::c(0.5) + d;
        r.s = i + (up ? 1 : 0) - 1;
        r.w[0] = A::c(0.5) * (a * a);
        r.w[1] = fma(-d, d, A::c(0.75));
        r.w[2] = A::c(0.5) * (b * b);
    } else {
        r.s = i - 1;
        cubic_weights<R>(A::from(f), r.w);
    }
    return r;
}

// node and half-node supports of one position (the half-node grid is shifted
// by +1/2 cell: Ex along x, etc.), and the cell floor(xi).  ec selects the
// energy-conserving half-node support: order ORDER - 1 (order 0: the nearest
// half node), stored with a zero last weight so that the interpolation code
// is shared.
template <int ORDER, class R>
__device__ __forceinline__ void supports(double xi, bool ec, Support<ORDER, R>& nd, Support<ORDER, R>& hf,
                                         int& cell) {
    using A = Arith<R>;
    double f;
    const int i = ifloor_frac(xi, f);
    cell = i;
    const bool up = ge_half(f);
    const R fr = A::from(f);
    if constexpr (ORDER == 1) {
        nd.s = i;
        nd.w[0] = A::c(1.0) - fr;
        nd.w[1] = fr;
        if (ec) {  // box shape: half node i (at i + 1/2) carries the point
            hf.s = i;
            hf.w[0] = A::c(1.0);
            hf.w[1] = A::c(0.0);
        } else {
            const R g = fr + (up ? A::c(-0.5) : A::c(0.5));  // xi - 1/2 - floor(xi - 1/2)
            hf.s = up ? i : i - 1;
            hf.w[0] = A::c(1.0) - g;
            hf.w[1] = g;
        }
    } else if constexpr (ORDER == 2) {
        const R d = up ? fr - A::c(1.0) : fr;  // node: xi - floor(xi + 1/2)
        const R a = A::c(0.5) - d, b = A::c(0.5) + d;
        nd.s = i + (up ? 1 : 0) - 1;
        nd.w[0] = A::c(0.5) * (a * a);
        nd.w[1] = fma(-d, d, A::c(0.75));
        nd.w[2] = A::c(0.5) * (b * b);
        if (ec) {  // hat on the half-node grid: g = frac(xi - 1/2)
            const R g = fr + (up ? A::c(-0.5) : A::c(0.5));
            hf.s = up ? i : i - 1;
            hf.w[0] = A::c(1.0) - g;
            hf.w[1] = g;
            hf.w[2] = A::c(0.0);
        } else {
            const R h = fr - A::c(0.5);  // half: (xi - 1/2) - floor(xi), nearest half-node floor(xi)
            const R ah = A::c(0.5) - h, bh = A::c(0.5) + h;
            hf.s = i - 1;
            hf.w[0] = A::c(0.5) * (ah * ah);
            hf.w[1] = fma(-h, h, A::c(0.75));
            hf.w[2] = A::c(0.5) * (bh * bh);
        }
    } else {
        nd.s = i - 1;
        cubic_weights<R>(fr, nd.w);
        if (ec) {  // quadratic on the half-node grid around the nearest half node floor(xi)
            const R h = fr - A::c(0.5);
            const R ah = A::c(0.5) - h, bh = A::c(0.5) + h;
            hf.s = i - 1;
            hf.w[0] = A::c(0.5) * (ah * ah);
            hf.w[1] = fma(-h, h, A::c(0.75));
            hf.w[2] = A::c(0.5) * (bh * bh);
            hf.w[3] = A::c(0.0);
        } else {
            const R g = fr + (up ? A::c(-0.5) : A::c(0.5));
            hf.s = (up ? i : i - 1) - 1;
            cubic_weights<R>(g, hf.w);
        }
    }
}

// supports relative to a tile origin o, from the global position: floor and
// fraction of x are those of x - o (o an integer), without forming x - o
template <int ORDER, class R>
__device__ __forceinline__ Support<ORDER, R> support_at(double x, int o) {
    Support<ORDER, R> r = support<ORDER, R>(x);
    r.s -= o;
    return r;
}
template <int ORDER, class R>
__device__ __forceinline__ void supports_at(double x, int o, bool ec, Support<ORDER, R>& nd,
                                            Support<ORDER, R>& hf, int& cell) {
    supports<ORDER, R>(x, ec, nd, hf, cell);
    nd.s -= o;
    hf.s -= o;
    cell -= o;
}

// E/B tile halo below the tile origin: 1 cell (orders 1, 2), 2 cells (order 3)
template <int ORDER>
struct EBHalo {
    static constexpr int lo = ORDER == 3 ? 2 : 1;
};

// interpolation of one component from a shared tile with extents (SX, SY);
// the tile holds R values (doubles, or float pairs converted in place).  D,
// when given (linear FP64), holds the tile's x differences F[x+1] - F[x] on
// rows of SX - 1, so that each x lerp is one FMA.
template <class R, int ORDER, int DIM>
__device__ __forceinline__ R interp(const R* __restrict__ F, int SX, int SY, const Support<ORDER, R>& sx,
                                    const Support<ORDER, R>& sy, const Support<ORDER, R>& sz,
                                    const R* __restrict__ D = nullptr) {
    // tile column 0 is local cell -EBHalo<ORDER>::lo
    constexpr int H = EBHalo<ORDER>::lo;
    if constexpr (ORDER == 1 && std::is_same<R, double>::value) {
        if (D) {
            auto lerp = [](R a, R b, R f) { return fma(f, b - a, a); };
            const R fx = sx.w[1];
            const int DX = SX - 1;
            if constexpr (DIM == 3) {
                const int r00 = (sz.s + H) * SY + (sy.s + H);
                const int x = sx.s + H;
                const R a00 = fma(fx, D[r00 * DX + x], F[r00 * SX + x]);
                const R a10 = fma(fx, D[(r00 + 1) * DX + x], F[(r00 + 1) * SX + x]);
                const R a01 = fma(fx, D[(r00 + SY) * DX + x], F[(r00 + SY) * SX + x]);
                const R a11 = fma(fx, D[(r00 + SY + 1) * DX + x], F[(r00 + SY + 1) * SX + x]);
                return lerp(lerp(a00, a10, sy.w[1]), lerp(a01, a11, sy.w[1]), sz.w[1]);
            } else {
                const int r0 = sz.s + H, x = sx.s + H;
                const R a0 = fma(fx, D[r0 * DX + x], F[r0 * SX + x]);
                const R a1 = fma(fx, D[(r0 + 1) * DX + x], F[(r0 + 1) * SX + x]);
                return lerp(a0, a1, sz.w[1]);
            }
        }
    }
    if constexpr (ORDER == 1) {
        // linear: nested lerps a + f (b - a) need only the fractional parts
        auto lerp = [](R a, R b, R f) { return fma(f, b - a, a); };
        const R fx = sx.w[1];
        if constexpr (DIM == 3) {
            const R* r00 = F + ((sz.s + H) * SY + (sy.s + H)) * SX + (sx.s + H);
            const R* r10 = r00 + SX;
            const R* r01 = r00 + SX * SY;
            const R* r11 = r01 + SX;
            const R a0 = lerp(lerp(r00[0], r00[1], fx), lerp(r10[0], r10[1], fx), sy.w[1]);
            const R a1 = lerp(lerp(r01[0], r01[1], fx), lerp(r11[0], r11[1], fx), sy.w[1]);
            return lerp(a0, a1, sz.w[1]);
        } else {
            const R* r0 = F + (sz.s + H) * SX + (sx.s + H);
            const R* r1 = r0 + SX;
            return lerp(lerp(r0[0], r0[1], fx), lerp(r1[0], r1[1], fx), sz.w[1]);
        }
    } else if constexpr (DIM == 3) {
        R acc;
#pragma unroll
        for (int c = 0; c <= ORDER; ++c) {
            R pl;
#pragma unroll
            for (int b = 0; b <= ORDER; ++b) {
                const R* row = F + ((sz.s + H + c) * SY + (sy.s + H + b)) * SX + (sx.s + H);
                R r = sx.w[0] * row[0];
#pragma unroll
                for (int a = 1; a <= ORDER; ++a) r = fma(sx.w[a], row[a], r);
                pl = (b == 0) ? sy.w[0] * r : fma(sy.w[b], r, pl);
            }
            acc = (c == 0) ? sz.w[0] * pl : fma(sz.w[c], pl, acc);
        }
        return acc;
    } else {
        R acc;
#pragma unroll
        for (int c = 0; c <= ORDER; ++c) {
            const R* row = F + (sz.s + H + c) * SX + (sx.s + H);
            R r = sx.w[0] * row[0];
#pragma unroll
            for (int a = 1; a <= ORDER; ++a) r = fma(sx.w[a], row[a], r);
            acc = (c == 0) ? sz.w[0] * r : fma(sz.w[c], r, acc);
        }
        return acc;
    }
}

template <class T>
__device__ __forceinline__ T pick3(int a, const T& v0, const T& v1, const T& v2) {
    return a == 0 ? v0 : (a == 1 ? v1 : v2);
}

// The six E/B components at one particle.  E_a sits on the half-node grid
// along a and on nodes across it, B_a the other way round.  FP64 and FP32
// unroll the six interpolations; float-float runs them as a loop (its operations are
// 7-11 FP32 instructions each, and six unrolled copies overflow the
// instruction cache).
template <class R, int ORDER, int DIM>
__device__ __forceinline__ void gather6(const R* __restrict__ sEB, int stride, int SX, int SY,
                                        const Support<ORDER, R>* nd, const Support<ORDER, R>* hf, R* e,
                                        R* b, const R* __restrict__ sD = nullptr, int dstride = 0) {
    if constexpr (!std::is_same<R, dd>::value) {
        const bool hd = sD != nullptr;
        e[0] = interp<R, ORDER, DIM>(sEB, SX, SY, hf[0], nd[1], nd[2], hd ? sD : nullptr);
        e[1] = interp<R, ORDER, DIM>(sEB + stride, SX, SY, nd[0], hf[1], nd[2], hd ? sD + dstride : nullptr);
        e[2] = interp<R, ORDER, DIM>(sEB + 2 * stride, SX, SY, nd[0], nd[1], hf[2], hd ? sD + 2 * dstride : nullptr);
        b[0] = interp<R, ORDER, DIM>(sEB + 3 * stride, SX, SY, nd[0], hf[1], hf[2], hd ? sD + 3 * dstride : nullptr);
        b[1] = interp<R, ORDER, DIM>(sEB + 4 * stride, SX, SY, hf[0], nd[1], hf[2], hd ? sD + 4 * dstride : nullptr);
        b[2] = interp<R, ORDER, DIM>(sEB + 5 * stride, SX, SY, hf[0], hf[1], nd[2], hd ? sD + 5 * dstride : nullptr);
    } else {
        R v0 = Arith<R>::c(0.0), v1 = v0, v2 = v0, v3 = v0, v4 = v0, v5 = v0;
#pragma unroll 1
        for (int c = 0; c < 6; ++c) {
            const int a = c < 3 ? c : c - 3;
            const bool isb = c >= 3;
            const Support<ORDER, R> sx = ((a == 0) != isb) ? hf[0] : nd[0];
            const Support<ORDER, R> sy = ((a == 1) != isb) ? hf[1] : nd[1];
            const Support<ORDER, R> sz = ((a == 2) != isb) ? hf[2] : nd[2];
            const R v = interp<R, ORDER, DIM>(sEB + c * stride, SX, SY, sx, sy, sz);
            v0 = c == 0 ? v : v0;
            v1 = c == 1 ? v : v1;
            v2 = c == 2 ? v : v2;
            v3 = c == 3 ? v : v3;
            v4 = c == 4 ? v : v4;
            v5 = c == 5 ? v : v5;
        }
        e[0] = v0; e[1] = v1; e[2] = v2;
        b[0] = v3; b[1] = v4; b[2] = v5;
    }
}

// Esirkepov node shapes on a common window of W nodes starting at the lower of
// the two supports: W = ORDER + 1 when the particle keeps its support (the
// in-cell case, most particles), W = ORDER + 2 when it moves to a neighbour.
template <int ORDER, int W, class R>
struct Window {
    int base;
    R S0[W];
    R DS[W];
};

template <int ORDER, int W, class R>
__device__ __forceinline__ bool make_window(const Support<ORDER, R>& a, const Support<ORDER, R>& b,
                                            Window<ORDER, W, R>& win) {
    int base = min(a.s, b.s);
    int oa = a.s - base, ob = b.s - base;
    if (oa > W - ORDER - 1 || ob > W - ORDER - 1) return false;
    win.base = base;
    const R zero = Arith<R>::c(0.0);
#pragma unroll
    for (int l = 0; l < W; ++l) {
        R s0 = zero, s1 = zero;
#pragma unroll
        for (int k = 0; k <= ORDER; ++k) {
            s0 = (l - oa == k) ? a.w[k] : s0;
            s1 = (l - ob == k) ? b.w[k] : s1;
        }
        win.S0[l] = s0;
        win.DS[l] = s1 - s0;
    }
    return true;
}

struct Tile {
    int sim;
    int t;
    int o[3];  // origin cell
};

__device__ __forceinline__ void tile_origin(const SimDev& S, int t, int o[3]) {
    int b = t / S.tiles_per_box, lt = t - b * S.tiles_per_box;
    int bx = b % S.nb[0], by = (b / S.nb[0]) % S.nb[1], bz = b / (S.nb[0] * S.nb[1]);
    int tx = lt % S.tpb[0], ty = (lt / S.tpb[0]) % S.tpb[1], tz = lt / (S.tpb[0] * S.tpb[1]);
    o[0] = bx * S.bsz[0] + tx * S.T[0];
    o[1] = by * S.bsz[1] + ty * S.T[1];
    o[2] = bz * S.bsz[2] + tz * S.T[2];
}

// tile key of a global cell (box-major numbering); SV: SimDev or HotSim
template <class SV>
__device__ __forceinline__ int tile_key(const SV& S, int ix, int iy, int iz) {
    int bx = ix / S.bsz[0], by = iy / S.bsz[1], bz = iz / S.bsz[2];
    int tx = (ix - bx * S.bsz[0]) / S.T[0];
    int ty = (iy - by * S.bsz[1]) / S.T[1];
    int tz = (iz - bz * S.bsz[2]) / S.T[2];
    int b = (bz * S.nb[1] + by) * S.nb[0] + bx;
    return b * S.tiles_per_box + (tz * S.tpb[1] + ty) * S.tpb[0] + tx;
}

__device__ __forceinline__ void warp_hist_add(int32_t* count, int key) {
    unsigned act = __activemask();
    unsigned peers = __match_any_sync(act, key);
    int lane = threadIdx.x & 31;
    if (lane == __ffs(peers) - 1) atomicAdd(count + key, __popc(peers));
}

// The fields of a simulation and of its species that the particle loop reads,
// staged in shared memory once per work unit.  Read from the SimDev in global
// memory they would be fetched again for every particle (the loop's stores to
// the particle arrays might alias them as far as the compiler can tell).
struct HotSp {
    double* cur[7];
    int32_t* key;
    int32_t* count;
};
struct HotSim {
    double nd[3];
    int T[3], n[3], bsz[3], nb[3], tpb[3], ebs[3];
    int tiles_per_box, ntiles, absorb, ec, jlo;
    HotSp sp[PIC_MAXSP];
};

__device__ __forceinline__ void stage_hot(HotSim& h, const SimDev& S) {
    for (int a = 0; a < 3; ++a) {
        h.nd[a] = S.nd[a];
        h.T[a] = S.T[a];
        h.n[a] = S.n[a];
        h.bsz[a] = S.bsz[a];
        h.nb[a] = S.nb[a];
        h.tpb[a] = S.tpb[a];
        h.ebs[a] = S.ebs[a];
    }
    h.tiles_per_box = S.tiles_per_box;
    h.ntiles = S.ntiles;
    h.absorb = S.absorb;
    h.ec = S.ec;
    h.jlo = S.jlo;
    for (int i = 0; i < S.nsp; ++i) {
        for (int a = 0; a < 7; ++a) h.sp[i].cur[a] = S.sp[i].cur[a];
        h.sp[i].key = S.sp[i].key;
        h.sp[i].count = S.sp[i].count;
    }
}

// Per-warp ring buffers of cell-crossing particles (struct of arrays, WQ
// slots per warp, up to 8 warps per CTA), in global scratch.
constexpr int WQ = 64;
constexpr int QMAXWARPS = 8;
// queue fields: 0 x^n, 1 z^n, 2 x^{n+1}, 3 z^{n+1} (global, unwrapped), 4 q w,
// 5 y^n (3D) or vy (2D), 6 y^{n+1} (3D)
template <int DIM>
struct QFields {
    static constexpr int n = DIM == 3 ? 7 : 6;
};

static_assert(QFields<3>::n * WQ == PIC_RING_DOUBLES && QMAXWARPS == 8,
              "a warp's global ring holds 7 fields of WQ slots; rings are allocated for 8 warps per CTA");

struct SmemPlan {
    int eb_stride;  // doubles per E/B component (multiple of 16 -> 128-byte aligned)
    int d_stride;   // doubles per component of the x-difference tile (0: none)
    int eb_vol, d_vol;
    int pb_off;     // doubles from the base to the particle staging buffers
    size_t bytes;
};

// Particle staging (FP32 variant): per warp two buffers of the 7 stored
// values of 32 particles, filled by cp.async one loop iteration ahead.
constexpr int PIN_SLOTS = 7 * 32;
constexpr int PIC_PBUF_DOUBLES = QMAXWARPS * 2 * PIN_SLOTS;

// xdiff: the x differences of the staged E/B tile are kept beside it (linear
// FP64).  pbuf: particle staging buffers (FP32 variant).  The FP32 variant
// converts the staged E/B tile in place: for linear shapes to float pairs
// (F[x], F[x+1] - F[x]), component c at pair c * eb_stride; otherwise to
// floats, component c at float c * eb_stride.
// Layout: E/B tile (TMA) | x differences | particle buffers.
__host__ __device__ inline SmemPlan smem_plan(const int ebs[3], bool xdiff, bool pbuf) {
    SmemPlan p;
    p.eb_vol = ebs[0] * ebs[1] * ebs[2];
    p.d_vol = xdiff ? (ebs[0] - 1) * ebs[1] * ebs[2] : 0;
    p.eb_stride = (p.eb_vol + 15) & ~15;
    p.d_stride = (p.d_vol + 15) & ~15;
    p.pb_off = 6 * p.eb_stride + 6 * p.d_stride;
    p.bytes = (size_t)(p.pb_off + (pbuf ? PIC_PBUF_DOUBLES : 0)) * sizeof(double);  // tiles and buffers
    return p;
}

// whether a precision / shape order keeps the x-difference tile: FP64 linear
__host__ __device__ inline bool uses_xdiff(int prec, int order) { return prec == 0 && order == 1; }

// double <-> float on the bit patterns without branches: magnitudes below
// 2^-100 (and zero) become a signed zero (an absolute error below 2^-100,
// far inside the FP32 variant's tolerance), larger ones round to 24 bits
__device__ __forceinline__ float f32_of(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned long long u = b & 0x7FFFFFFFFFFFFFFFull;
    const unsigned sgn = (unsigned)(b >> 32) & 0x80000000u;
    const unsigned m = (unsigned)(((u + (1ull << 28)) >> 29) - (896ull << 23));
    return __uint_as_float(sgn | ((u >> 52) >= 1023 - 100 ? m : 0u));
}
__device__ __forceinline__ double f64_of(float f) {
    const unsigned b = __float_as_uint(f), a = b & 0x7FFFFFFFu;
    const unsigned long long sg = (unsigned long long)(b & 0x80000000u) << 32;
    const unsigned long long m = ((unsigned long long)a + (896ull << 23)) << 29;
    return __longlong_as_double((long long)(sg | (a >= 0x00800000u ? m : 0ull)));
}

// Current accumulation.  Every precision adds each contribution to the
// global FP64 J with red.global.add.f64: the add runs in L2, nothing returns
// to the SM, and no FP64 instruction is spent on it.  (A shared-memory FP64
// atomic is a compare-and-swap loop whose retries each cost a full-warp FP64
// add; a shared FP32 atomic add is a compare-and-swap loop as well, measured
// at about 2.3 tries per add on the foil, and moving the FP32 variant's
// current from a shared FP32 tile to these reductions took its particle
// kernel from 895 to 696 us on the 128^3 foil.)  A float-float value is
// renormalised and merged to one double first; an FP32 value is widened on its
// bit pattern (subnormal floats, below 2^-126, become zero).
__device__ __forceinline__ void red_f64(double* p, double v) {
    asm volatile("red.global.add.f64 [%0], %1;" ::"l"(__cvta_generic_to_global(p)), "d"(v) : "memory");
}
__device__ __forceinline__ void jadd(double* p, double v) { red_f64(p, v); }
__device__ __forceinline__ void jadd(double* p, dd v) { red_f64(p, dd_to_norm(v)); }
__device__ __forceinline__ void jadd(double* p, float v) { red_f64(p, f64_of(v)); }

// Where a tile's current goes: base points at component 0 of local node
// (-jlo, -jlo, -jlo) of the tile (jlo = S.jlo; y is 0 in 2D) in the padded J
// arrays, cs is the component stride, sy and sz the row and plane strides.
// The guard cells (2 to 4 per side) hold the contributions that fall outside
// the domain until the fold kernel adds them to their periodic images.
struct JView {
    double* base;
    int64_t cs;
    int sy, sz;
};

// Esirkepov deposit of one particle into the J arrays (view V) on windows of
// W nodes per direction.  n*: node supports at x^n, m*: at x^{n+1} (local cells).
// Prefix sums of DS along each current's own direction times the transverse
// weight S0a S0b + DSa S0b/2 + S0a DSb/2 + DSa DSb/3 = A_a A_b + DS_a DS_b / 12
// with A = S0 + DS/2.  qw and vy in R; the prefactors -1/(dA dt) come from jf.
template <class R, int DIM, int ORDER, int W, class SV>
__device__ __forceinline__ bool deposit(const SV& S, const JView& V,
                                        R qw, R vy, const R* jf, const Support<ORDER, R>& n0,
                                        const Support<ORDER, R>& n1, const Support<ORDER, R>& n2,
                                        const Support<ORDER, R>& m0, const Support<ORDER, R>& m1,
                                        const Support<ORDER, R>& m2) {
    using A = Arith<R>;
    Window<ORDER, W, R> wx, wy, wz;
    bool ok = make_window<ORDER, W, R>(n0, m0, wx) && make_window<ORDER, W, R>(n2, m2, wz);
    if (DIM == 3) ok = ok && make_window<ORDER, W, R>(n1, m1, wy);
    if (!ok) return false;
    const int sy = V.sy, sz = V.sz, lo = S.jlo;
    double* Jx = V.base;
    double* Jy = V.base + V.cs;
    double* Jz = V.base + 2 * V.cs;
    const R half = A::c(0.5), k12 = A::c(1.0 / 12.0);
    R Ax[W], Az[W], Dx12[W], Dz12[W];
#pragma unroll
    for (int l = 0; l < W; ++l) {
        Ax[l] = fma(half, wx.DS[l], wx.S0[l]);
        Az[l] = fma(half, wz.DS[l], wz.S0[l]);
        Dx12[l] = k12 * wx.DS[l];
        Dz12[l] = k12 * wz.DS[l];
    }
    if constexpr (DIM == 3 && std::is_same<R, dd>::value) {
        // float-float: one loop over the three currents (prefix axis a,
        // transverse axes b < c), to keep the code small
        R Ay[W], Dy12[W];
#pragma unroll
        for (int l = 0; l < W; ++l) {
            Ay[l] = fma(half, wy.DS[l], wy.S0[l]);
            Dy12[l] = k12 * wy.DS[l];
        }
        double* origin = V.base + (wz.base + lo) * sz + (wy.base + lo) * sy + (wx.base + lo);
#pragma unroll 1
        for (int a = 0; a < 3; ++a) {
            const int b = a == 0 ? 1 : 0, c = a == 2 ? 1 : 2;
            const int sa = pick3(a, 1, sy, sz), sb = pick3(b, 1, sy, sz), sc = pick3(c, 1, sy, sz);
            const R cf = qw * pick3(a, jf[0], jf[1], jf[2]);
            R Pf[W - 1], Ab[W], Ac[W], Db[W], Dc12[W];
            R acc = A::c(0.0);
#pragma unroll
            for (int l = 0; l < W; ++l) {
                if (l < W - 1) {
                    acc = acc + pick3(a, wx.DS[l], wy.DS[l], wz.DS[l]);
                    Pf[l] = cf * acc;
                }
                Ab[l] = b == 0 ? Ax[l] : Ay[l];
                Db[l] = b == 0 ? wx.DS[l] : wy.DS[l];
                Ac[l] = c == 1 ? Ay[l] : Az[l];
                Dc12[l] = c == 1 ? Dy12[l] : Dz12[l];
            }
            double* Ja = origin + a * V.cs;
#pragma unroll 1
            for (int k = 0; k < W; ++k) {
                R ack = Ac[0], dck = Dc12[0];
#pragma unroll
                for (int q = 1; q < W; ++q) {
                    ack = k == q ? Ac[q] : ack;
                    dck = k == q ? Dc12[q] : dck;
                }
#pragma unroll
                for (int j = 0; j < W; ++j) {
                    const R T = fma(Ab[j], ack, Db[j] * dck);
                    double* row = Ja + k * sc + j * sb;
#pragma unroll
                    for (int l = 0; l < W - 1; ++l) jadd(row + l * sa, Pf[l] * T);
                }
            }
        }
    } else if constexpr (DIM == 3) {
        R Ay[W];
#pragma unroll
        for (int l = 0; l < W; ++l) Ay[l] = fma(half, wy.DS[l], wy.S0[l]);
        const int bx = wx.base + lo, by = wy.base + lo, bz = wz.base + lo;
        {
            const R c = qw * jf[0];
            R Pf[W - 1];
            R acc = A::c(0.0);
#pragma unroll
            for (int l = 0; l < W - 1; ++l) { acc = acc + wx.DS[l]; Pf[l] = c * acc; }
#pragma unroll
            for (int k = 0; k < W; ++k)
#pragma unroll
                for (int j = 0; j < W; ++j) {
                    const R T = fma(Ay[j], Az[k], wy.DS[j] * Dz12[k]);
                    double* row = Jx + (bz + k) * sz + (by + j) * sy + bx;
#pragma unroll
                    for (int l = 0; l < W - 1; ++l) jadd(row + l, Pf[l] * T);
                }
        }
        {
            const R c = qw * jf[1];
            R Pf[W - 1];
            R acc = A::c(0.0);
#pragma unroll
            for (int j = 0; j < W - 1; ++j) { acc = acc + wy.DS[j]; Pf[j] = c * acc; }
#pragma unroll
            for (int k = 0; k < W; ++k)
#pragma unroll
                for (int i = 0; i < W; ++i) {
                    const R T = fma(Ax[i], Az[k], wx.DS[i] * Dz12[k]);
                    double* col = Jy + (bz + k) * sz + by * sy + (bx + i);
#pragma unroll
                    for (int j = 0; j < W - 1; ++j) jadd(col + j * sy, Pf[j] * T);
                }
        }
        {
            const R c = qw * jf[2];
            R Pf[W - 1];
            R acc = A::c(0.0);
#pragma unroll
            for (int k = 0; k < W - 1; ++k) { acc = acc + wz.DS[k]; Pf[k] = c * acc; }
#pragma unroll
            for (int j = 0; j < W; ++j)
#pragma unroll
                for (int i = 0; i < W; ++i) {
                    const R T = fma(Ax[i], Ay[j], Dx12[i] * wy.DS[j]);
                    double* col = Jz + bz * sz + (by + j) * sy + (bx + i);
#pragma unroll
                    for (int k = 0; k < W - 1; ++k) jadd(col + k * sz, Pf[k] * T);
                }
        }
    } else {
        const int bx = wx.base + lo, bz = wz.base + lo;
        {  // Jx(i,k) = -(q w /(dz dt)) sum_{i'<=i} DSx(i') (S0z + DSz/2)
            const R c = qw * jf[0];
            R Pf[W - 1];
            R acc = A::c(0.0);
#pragma unroll
            for (int l = 0; l < W - 1; ++l) { acc = acc + wx.DS[l]; Pf[l] = c * acc; }
#pragma unroll
            for (int k = 0; k < W; ++k) {
                double* row = Jx + (bz + k) * sz + bx;
#pragma unroll
                for (int l = 0; l < W - 1; ++l) jadd(row + l, Pf[l] * Az[k]);
            }
        }
        {
            const R c = qw * jf[2];
            R Pf[W - 1];
            R acc = A::c(0.0);
#pragma unroll
            for (int k = 0; k < W - 1; ++k) { acc = acc + wz.DS[k]; Pf[k] = c * acc; }
#pragma unroll
            for (int i = 0; i < W; ++i) {
                double* col = Jz + bz * sz + (bx + i);
#pragma unroll
                for (int k = 0; k < W - 1; ++k) jadd(col + k * sz, Pf[k] * Ax[i]);
            }
        }
        {  // out-of-plane Jy = q w vy / (dx dz) * (Ax Az + DSx DSz / 12)
            const R c = qw * vy * jf[1];
#pragma unroll
            for (int k = 0; k < W; ++k)
#pragma unroll
                for (int i = 0; i < W; ++i)
                    jadd(Jy + (bz + k) * sz + (bx + i), c * fma(Ax[i], Az[k], Dx12[i] * wz.DS[k]));
        }
    }
    return true;
}

// Linear shapes, particle keeping its cell in every direction: the window is
// the two nodes of the cell, DS = (-d, d) with d = f1 - f0, so the prefix sum
// has one term and the transverse weight A_a A_b + DS_a DS_b / 12 is
// A_a A_b +- d_a d_b / 12 (A = (1 - m, m), m = f0 + d/2).  Same weights as
// deposit<R, DIM, 1, 2>, with fewer instructions.
template <class R, int DIM, class SV>
__device__ __forceinline__ void deposit_lin_incell_d(const SV& S, const JView& V,
                                                     R qw, R vy, const R* jf, const Support<1, R>* n,
                                                     const R* disp);

template <class R, int DIM, class SV>
__device__ __forceinline__ void deposit_lin_incell(const SV& S, const JView& V,
                                                   R qw, R vy, const R* jf,
                                                   const Support<1, R>* n, const Support<1, R>* m) {
    const R disp[3] = {m[0].w[1] - n[0].w[1], m[1].w[1] - n[1].w[1], m[2].w[1] - n[2].w[1]};
    deposit_lin_incell_d<R, DIM, SV>(S, V, qw, vy, jf, n, disp);
}

// the same deposit, given the in-cell displacement disp[a] = x^{n+1} - x^n
// (cells) of each direction
template <class R, int DIM, class SV>
__device__ __forceinline__ void deposit_lin_incell_d(const SV& S, const JView& V,
                                                     R qw, R vy, const R* jf, const Support<1, R>* n,
                                                     const R* disp) {
    using A = Arith<R>;
    const R k12 = A::c(1.0 / 12.0), half = A::c(0.5), one = A::c(1.0);
    const int sy = V.sy, sz = V.sz, lo = S.jlo;
    double* Jx = V.base;
    double* Jy = V.base + V.cs;
    double* Jz = V.base + 2 * V.cs;
    const R dx = disp[0], dz = disp[2];
    const R mx = fma(half, dx, n[0].w[1]), mz = fma(half, dz, n[2].w[1]);
    const R ax0 = one - mx, az0 = one - mz;
    const int bx = n[0].s + lo, bz = n[2].s + lo;
    if constexpr (DIM == 3 && std::is_same<R, dd>::value) {
        // float-float: one loop over the three currents (axis a, transverse b < c)
        const R dy = disp[1];
        const R my = fma(half, dy, n[1].w[1]);
        const R ay0 = one - my;
        const int by = n[1].s + lo;
        double* origin = V.base + bz * sz + by * sy + bx;
#pragma unroll 1
        for (int a = 0; a < 3; ++a) {
            const int b = a == 0 ? 1 : 0, c = a == 2 ? 1 : 2;
            const int sb = pick3(b, 1, sy, sz), sc = pick3(c, 1, sy, sz);
            const R db = b == 0 ? dx : dy, dc = c == 1 ? dy : dz;
            const R mb = b == 0 ? mx : my, mc = c == 1 ? my : mz;
            const R ab = b == 0 ? ax0 : ay0, ac = c == 1 ? ay0 : az0;
            const R e = (db * dc) * k12;
            const R pf = -((qw * pick3(a, jf[0], jf[1], jf[2])) * pick3(a, dx, dy, dz));
            double* r = origin + a * V.cs;
            jadd(r, pf * fma(ab, ac, e));
            jadd(r + sb, pf * fma(mb, ac, -e));
            jadd(r + sc, pf * fma(ab, mc, -e));
            jadd(r + sb + sc, pf * fma(mb, mc, e));
        }
    } else if constexpr (DIM == 3) {
        // value of node (b, c) of current a: pf_a (A_b A_c + s d_b d_c / 12),
        // s = +1 on the diagonal nodes, -1 off it, pf_a = -q w jf_a d_a; with
        // pe_a = pf_a d_b d_c / 12 = -q w jf_a (d_x d_y d_z / 12) and the node
        // weights (1 - m, m) each value is one FMA of pf_a A_b against A_c
        const R dy = disp[1];
        const R my = fma(half, dy, n[1].w[1]);
        const R ay0 = one - my;
        const int by = n[1].s + lo;
        const R d3 = (dx * dy) * (dz * k12);
        {   // Jx at (bx, by + j, bz + k)
            const R q = qw * jf[0];
            const R pf = -(q * dx), pe = -(q * d3);
            const R p1 = pf * my, p0 = pf - p1;
            double* r = Jx + bz * sz + by * sy + bx;
            jadd(r, fma(p0, az0, pe));
            jadd(r + sy, fma(p1, az0, -pe));
            jadd(r + sz, fma(p0, mz, -pe));
            jadd(r + sz + sy, fma(p1, mz, pe));
        }
        {   // Jy at (bx + i, by, bz + k)
            const R q = qw * jf[1];
            const R pf = -(q * dy), pe = -(q * d3);
            const R p1 = pf * mx, p0 = pf - p1;
            double* r = Jy + bz * sz + by * sy + bx;
            jadd(r, fma(p0, az0, pe));
            jadd(r + 1, fma(p1, az0, -pe));
            jadd(r + sz, fma(p0, mz, -pe));
            jadd(r + sz + 1, fma(p1, mz, pe));
        }
        {   // Jz at (bx + i, by + j, bz)
            const R q = qw * jf[2];
            const R pf = -(q * dz), pe = -(q * d3);
            const R p1 = pf * mx, p0 = pf - p1;
            double* r = Jz + bz * sz + by * sy + bx;
            jadd(r, fma(p0, ay0, pe));
            jadd(r + 1, fma(p1, ay0, -pe));
            jadd(r + sy, fma(p0, my, -pe));
            jadd(r + sy + 1, fma(p1, my, pe));
        }
    } else {
        {   // Jx at (bx, bz + k): -(q w/(dz dt)) DSx A_z
            const R pf = -((qw * jf[0]) * dx);
            double* r = Jx + bz * sz + bx;
            jadd(r, pf * az0);
            jadd(r + sz, pf * mz);
        }
        {   // Jz at (bx + i, bz)
            const R pf = -((qw * jf[2]) * dz);
            double* r = Jz + bz * sz + bx;
            jadd(r, pf * ax0);
            jadd(r + 1, pf * mx);
        }
        {   // out-of-plane Jy at (bx + i, bz + k)
            const R e = (dx * dz) * k12;
            const R c = qw * vy * jf[1];
            double* r = Jy + bz * sz + bx;
            jadd(r, c * fma(ax0, az0, e));
            jadd(r + 1, c * fma(mx, az0, -e));
            jadd(r + sz, c * fma(ax0, mz, -e));
            jadd(r + sz + 1, c * fma(mx, mz, e));
        }
    }
}

// One particle's stored state as read from HBM (positions in global cell
// units, momenta and weight as stored); loaded ahead of its push so that the
// loads of several particles per thread can be in flight together.
struct PIn {
    double X, Y, Z, u0, u1, u2, w;
};

template <int DIM, class SPV>
__device__ __forceinline__ PIn load_one(const SPV& sp, int64_t p) {
    PIn in;
    in.X = sp.cur[0][p];
    in.Y = (DIM == 3) ? sp.cur[1][p] : 0.0;
    in.Z = sp.cur[2][p];
    in.u0 = sp.cur[3][p];
    in.u1 = sp.cur[4][p];
    in.u2 = sp.cur[5][p];
    in.w = sp.cur[6][p];
    return in;
}

// The same values staged through shared memory: the lane's column of a
// staging buffer (value a of the particle at slot[32 a]), filled by cp.async
template <int DIM, class SPV>
__device__ __forceinline__ void stage_in(const SPV& sp, int64_t p, double* slot) {
#pragma unroll
    for (int a = 0; a < 7; ++a)
        if (DIM == 3 || a != 1) cp_async_8(slot + 32 * a, sp.cur[a] + p);
}
template <int DIM>
__device__ __forceinline__ PIn read_staged(const double* slot) {
    PIn in;
    in.X = slot[0];
    in.Y = (DIM == 3) ? slot[32] : 0.0;
    in.Z = slot[64];
    in.u0 = slot[96];
    in.u1 = slot[128];
    in.u2 = slot[160];
    in.w = slot[192];
    return in;
}

// Gather, Boris push, and deposit of one particle.  Particles that keep their
// support in every direction deposit at once on the small window; the others
// go to the warp's ring buffer, drained 32 at a time by drain_warp.
template <class R, int DIM, int ORDER, class SV, class SPV>
__device__ __forceinline__ void push_one(const SV& S, const SPV& sp, const Tile& tl,
                                         const R* __restrict__ sEB, const R* __restrict__ sD,
                                         const JView& V,
                                         double* __restrict__ sQw, unsigned* s_tail, const SmemPlan& P,
                                         const R* jf, const R* dtd, R kq, R qs, int64_t p, const PIn& in,
                                         int32_t* err) {
    using A = Arith<R>;
    double X = in.X, Z = in.Z;
    double Y = (DIM == 3) ? in.Y : 0.0;
    const R u0 = A::from(in.u0), u1 = A::from(in.u1), u2 = A::from(in.u2);
    const R qw = qs * A::from(in.w);

    // ---- gather at x^n: node and half-node supports per direction (tile-local nodes)
    Support<ORDER, R> nd[3], hf[3];
    int cx, cy = 0, cz;
    const bool ec = S.ec != 0;
    supports_at<ORDER, R>(X, tl.o[0], ec, nd[0], hf[0], cx);
    supports_at<ORDER, R>(Z, tl.o[2], ec, nd[2], hf[2], cz);
    if (DIM == 3) {
        supports_at<ORDER, R>(Y, tl.o[1], ec, nd[1], hf[1], cy);
    } else {
        nd[1].s = -1;
        nd[1].w[0] = A::c(1.0);
        hf[1] = nd[1];
    }
    {
        // the particle must sit in its tile (local cell index in [0, T)); the
        // E/B halo then covers every support above
        bool in = cx >= 0 && cx < S.T[0] && cz >= 0 && cz < S.T[2];
        if (DIM == 3) in = in && cy >= 0 && cy < S.T[1];
        if (!in) {
            atomicOr(err, PIC_DERR_BOUNDS);
            sp.key[p] = S.ntiles;
            warp_hist_add(sp.count, S.ntiles);
            return;
        }
    }
    const int SX = S.ebs[0], SY = S.ebs[1];
    R ev[3], bv[3];
    gather6<R, ORDER, DIM>(sEB, P.eb_stride, SX, SY, nd, hf, ev, bv, sD, P.d_stride);
    const R e0 = ev[0], e1 = ev[1], e2 = ev[2], b0 = bv[0], b1 = bv[1], b2 = bv[2];

    // ---- relativistic Boris push
    const R one = A::c(1.0);
    const R m0 = fma(kq, e0, u0), m1 = fma(kq, e1, u1), m2 = fma(kq, e2, u2);
    const R ig = A::rsqrt(fma(m2, m2, fma(m1, m1, fma(m0, m0, one))));
    const R kg = kq * ig;
    const R t0 = kg * b0, t1 = kg * b1, t2 = kg * b2;
    const R t2n = fma(t2, t2, fma(t1, t1, t0 * t0));
    const R sf = A::two_over(one + t2n);
    const R s0 = sf * t0, s1 = sf * t1, s2 = sf * t2;
    // u' = u- + u- x t, u+ = u- + u' x s, each component as two FMAs
    const R d0 = fma(m1, t2, fma(-m2, t1, m0));
    const R d1 = fma(m2, t0, fma(-m0, t2, m1));
    const R d2 = fma(m0, t1, fma(-m1, t0, m2));
    const R p0 = fma(d1, s2, fma(-d2, s1, m0));
    const R p1 = fma(d2, s0, fma(-d0, s2, m1));
    const R p2 = fma(d0, s1, fma(-d1, s0, m2));
    const R n0 = fma(kq, e0, p0), n1 = fma(kq, e1, p1), n2 = fma(kq, e2, p2);
    const R ign = A::rsqrt(fma(n2, n2, fma(n1, n1, fma(n0, n0, one))));
    const R v1 = n1 * ign;
    const double dX = A::to((n0 * ign) * dtd[0]), dZ = A::to((n2 * ign) * dtd[2]);
    const double dY = (DIM == 3) ? A::to(v1 * dtd[1]) : 0.0;

    // ---- Esirkepov deposit of J^{n+1/2} from x^n to x^{n+1}
    const double X1 = X + dX, Z1 = Z + dZ;
    const double Y1 = (DIM == 3) ? Y + dY : 0.0;
    Support<ORDER, R> mv[3];
    mv[0] = support_at<ORDER, R>(X1, tl.o[0]);
    mv[2] = support_at<ORDER, R>(Z1, tl.o[2]);
    if (DIM == 3) mv[1] = support_at<ORDER, R>(Y1, tl.o[1]);
    else mv[1] = nd[1];
    bool same = mv[0].s == nd[0].s && mv[2].s == nd[2].s && (DIM == 2 || mv[1].s == nd[1].s);
    if (same) {
        if constexpr (ORDER == 1)
            deposit_lin_incell<R, DIM, SV>(S, V, qw, v1, jf, nd, mv);
        else
            deposit<R, DIM, ORDER, ORDER + 1>(S, V, qw, v1, jf, nd[0], nd[1], nd[2], mv[0], mv[1], mv[2]);
    } else {
        // the ring never holds more than 31 + 32 entries: the warp drains 32
        // whenever 32 are waiting
        const unsigned slot = atomicAdd(s_tail, 1u) & (WQ - 1);
        sQw[0 * WQ + slot] = X;
        sQw[1 * WQ + slot] = Z;
        sQw[2 * WQ + slot] = X1;
        sQw[3 * WQ + slot] = Z1;
        sQw[4 * WQ + slot] = A::to(qw);
        sQw[5 * WQ + slot] = DIM == 3 ? Y : A::to(v1);
        if (DIM == 3) sQw[6 * WQ + slot] = Y1;
    }

    // ---- new position, boundary, re-sort key
    X = X1;
    Z = Z1;
    if (is_neg(X) || ge_pos(X, S.nd[0])) X = wrap_periodic(X, S.nd[0]);
    if (DIM == 3) {
        Y = Y1;
        if (is_neg(Y) || ge_pos(Y, S.nd[1])) Y = wrap_periodic(Y, S.nd[1]);
    }
    int key = -1;
    if (S.absorb > 0) {
        // z < A or z >= n - A for integer bounds: compare floor(z)
        const int iz = ifloor(Z);
        if (iz < S.absorb || iz >= S.n[2] - S.absorb) key = S.ntiles;
    } else {
        if (is_neg(Z) || ge_pos(Z, S.nd[2])) Z = wrap_periodic(Z, S.nd[2]);
    }
    if (key < 0) {
        int ix = min(max(ifloor(X), 0), S.n[0] - 1);
        int iy = (DIM == 3) ? min(max(ifloor(Y), 0), S.n[1] - 1) : 0;
        int iz = min(max(ifloor(Z), 0), S.n[2] - 1);
        // most particles stay in their tile: its key without the divisions
        bool own = (unsigned)(ix - tl.o[0]) < (unsigned)S.T[0] && (unsigned)(iz - tl.o[2]) < (unsigned)S.T[2];
        if (DIM == 3) own = own && (unsigned)(iy - tl.o[1]) < (unsigned)S.T[1];
        key = own ? tl.t : tile_key(S, ix, iy, iz);
    }
    sp.cur[0][p] = X;
    if (DIM == 3) sp.cur[1][p] = Y;
    sp.cur[2][p] = Z;
    sp.cur[3][p] = A::to(n0);
    sp.cur[4][p] = A::to(n1);
    sp.cur[5][p] = A::to(n2);
    sp.key[p] = key;
    warp_hist_add(sp.count, key);
}

// ---- FP32 variant, linear shapes: positions in 24-bit fixed point --------
// Adding M = 1.5 * 2^28 to a position X (cells, |X| < 2^27), rounded toward
// -infinity, truncates it to a multiple of 2^-24 and leaves it, as a
// fixed-point number with 24 fractional bits, in the low bits of the sum: one
// FP64 add gives the cell (the bits above 24: floor(X) exactly, negative X
// too) and the in-cell offset (the low 24) with integer instructions and no
// branches.  The move is carried in the same units (d rounded to 2^-24 of a
// cell), so the cell test of x^{n+1}, the in-cell displacement used by the
// deposit and the stored FP64 position agree exactly; after the first step
// every stored position lies on the 2^-24 grid.
constexpr double kFixM = 402653184.0;  // 1.5 * 2^28: ulp 2^-24 over [2^28, 2^29)
__device__ __forceinline__ long long fix24(double x) {
    return __double_as_longlong(__dadd_rd(x, kFixM)) - __double_as_longlong(kFixM);
}
__device__ __forceinline__ double unfix24(long long b) {
    return __longlong_as_double(b + __double_as_longlong(kFixM)) - kFixM;  // exact
}
__device__ __forceinline__ float frac24(long long b) { return (float)(int)(b & 0xFFFFFFll) * 5.9604644775390625e-8f; }

// Linear FP32 gather from the staged tile held as pairs (F[x], F[x+1] - F[x])
// of floats: each x lerp is one 8-byte shared load and one FMA, and gives the
// same float as a + f (b - a) on the two floats.  Component c starts at pair
// c * stride.
template <int DIM>
__device__ __forceinline__ float interp_pairs(const float2* __restrict__ F, int SX, int SY, const Support<1, float>& sx,
                                              const Support<1, float>& sy, const Support<1, float>& sz) {
    constexpr int H = EBHalo<1>::lo;
    auto lerp = [](float a, float b, float f) { return fmaf(f, b - a, a); };
    const float fx = sx.w[1];
    if constexpr (DIM == 3) {
        const float2* r = F + ((sz.s + H) * SY + (sy.s + H)) * SX + (sx.s + H);
        const float2 p00 = r[0], p10 = r[SX], p01 = r[SX * SY], p11 = r[SX * SY + SX];
        const float a00 = fmaf(fx, p00.y, p00.x), a10 = fmaf(fx, p10.y, p10.x);
        const float a01 = fmaf(fx, p01.y, p01.x), a11 = fmaf(fx, p11.y, p11.x);
        return lerp(lerp(a00, a10, sy.w[1]), lerp(a01, a11, sy.w[1]), sz.w[1]);
    } else {
        const float2* r = F + (sz.s + H) * SX + (sx.s + H);
        const float2 p0 = r[0], p1 = r[SX];
        return lerp(fmaf(fx, p0.y, p0.x), fmaf(fx, p1.y, p1.x), sz.w[1]);
    }
}
template <int DIM>
__device__ __forceinline__ void gather6_pairs(const float2* __restrict__ sP, int stride, int SX, int SY,
                                              const Support<1, float>* nd, const Support<1, float>* hf, float* e,
                                              float* b) {
    e[0] = interp_pairs<DIM>(sP, SX, SY, hf[0], nd[1], nd[2]);
    e[1] = interp_pairs<DIM>(sP + stride, SX, SY, nd[0], hf[1], nd[2]);
    e[2] = interp_pairs<DIM>(sP + 2 * stride, SX, SY, nd[0], nd[1], hf[2]);
    b[0] = interp_pairs<DIM>(sP + 3 * stride, SX, SY, nd[0], hf[1], hf[2]);
    b[1] = interp_pairs<DIM>(sP + 4 * stride, SX, SY, hf[0], nd[1], hf[2]);
    b[2] = interp_pairs<DIM>(sP + 5 * stride, SX, SY, hf[0], hf[1], nd[2]);
}

// gather, Boris push and deposit of one particle, FP32 arithmetic, linear shapes
template <int DIM, class SV, class SPV>
__device__ __forceinline__ void push_one_f32lin(const SV& S, const SPV& sp, const Tile& tl,
                                                const float* __restrict__ sEB, const JView& V,
                                                double* __restrict__ sQw, unsigned* s_tail, const SmemPlan& P,
                                                const float* jf, const float* dtd, float kq, float qs,
                                                int64_t p, const PIn& in, int32_t* err) {
    using A = Arith<float>;
    const double Xs[3] = {in.X, DIM == 3 ? in.Y : 0.0, in.Z};
    long long b0[3];
    int c[3];
    float f[3];
    bool inside = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (DIM == 2 && a == 1) {
            b0[a] = 0;
            c[a] = 0;
            f[a] = 0.0f;
            continue;
        }
        b0[a] = fix24(Xs[a]);
        c[a] = (int)(b0[a] >> 24) - tl.o[a];
        f[a] = frac24(b0[a]);
        inside = inside && (unsigned)c[a] < (unsigned)S.T[a];
    }
    if (!inside) {
        atomicOr(err, PIC_DERR_BOUNDS);
        sp.key[p] = S.ntiles;
        warp_hist_add(sp.count, S.ntiles);
        return;
    }
    // node supports (start c, weight f of the upper node) and half-node ones
    Support<1, float> nd[3], hf[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (DIM == 2 && a == 1) {
            nd[1].s = -1;
            nd[1].w[0] = 1.0f;
            nd[1].w[1] = 0.0f;
            hf[1] = nd[1];
            continue;
        }
        nd[a].s = c[a];
        nd[a].w[1] = f[a];
        const bool up = f[a] >= 0.5f;
        if (S.ec) {
            hf[a].s = c[a];
            hf[a].w[1] = 0.0f;
        } else {
            hf[a].s = up ? c[a] : c[a] - 1;
            hf[a].w[1] = f[a] + (up ? -0.5f : 0.5f);
        }
    }
    float ev[3], bv[3];
    gather6_pairs<DIM>(reinterpret_cast<const float2*>(sEB), P.eb_stride, S.ebs[0], S.ebs[1], nd, hf, ev, bv);
    const float u0 = f32_of(in.u0), u1 = f32_of(in.u1), u2 = f32_of(in.u2);
    const float qw = qs * f32_of(in.w);

    // relativistic Boris push
    const float m0 = fmaf(kq, ev[0], u0), m1 = fmaf(kq, ev[1], u1), m2 = fmaf(kq, ev[2], u2);
    const float ig = rsqrtf(fmaf(m2, m2, fmaf(m1, m1, fmaf(m0, m0, 1.0f))));
    const float kg = kq * ig;
    const float t0 = kg * bv[0], t1 = kg * bv[1], t2 = kg * bv[2];
    const float sf = 2.0f * __frcp_rn(1.0f + fmaf(t2, t2, fmaf(t1, t1, t0 * t0)));
    const float s0 = sf * t0, s1 = sf * t1, s2 = sf * t2;
    const float d0 = fmaf(m1, t2, fmaf(-m2, t1, m0));
    const float d1 = fmaf(m2, t0, fmaf(-m0, t2, m1));
    const float d2 = fmaf(m0, t1, fmaf(-m1, t0, m2));
    const float p0 = fmaf(d1, s2, fmaf(-d2, s1, m0));
    const float p1 = fmaf(d2, s0, fmaf(-d0, s2, m1));
    const float p2 = fmaf(d0, s1, fmaf(-d1, s0, m2));
    const float n0 = fmaf(kq, ev[0], p0), n1 = fmaf(kq, ev[1], p1), n2 = fmaf(kq, ev[2], p2);
    const float ign = rsqrtf(fmaf(n2, n2, fmaf(n1, n1, fmaf(n0, n0, 1.0f))));
    const float v1 = n1 * ign;
    const float dv[3] = {(n0 * ign) * dtd[0], DIM == 3 ? v1 * dtd[1] : 0.0f, (n2 * ign) * dtd[2]};

    // x^{n+1} in the same fixed point; in-cell test and displacement
    long long b1[3];
    float disp[3];
    bool same = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (DIM == 2 && a == 1) {
            b1[a] = 0;
            disp[a] = 0.0f;
            continue;
        }
        const int di = __float2int_rn(dv[a] * 16777216.0f);
        b1[a] = b0[a] + di;
        disp[a] = (float)di * 5.9604644775390625e-8f;
        same = same && (b1[a] >> 24) == (b0[a] >> 24);
    }
    if (same) {
        deposit_lin_incell_d<float, DIM, SV>(S, V, qw, v1, jf, nd, disp);
    } else {
        const unsigned slot = atomicAdd(s_tail, 1u) & (WQ - 1);
        sQw[0 * WQ + slot] = Xs[0];
        sQw[1 * WQ + slot] = Xs[2];
        sQw[2 * WQ + slot] = unfix24(b1[0]);
        sQw[3 * WQ + slot] = unfix24(b1[2]);
        sQw[4 * WQ + slot] = f64_of(qw);
        sQw[5 * WQ + slot] = DIM == 3 ? Xs[1] : f64_of(v1);
        if (DIM == 3) sQw[6 * WQ + slot] = unfix24(b1[1]);
    }

    // new position, boundary, re-sort key
    double X = unfix24(b1[0]), Y = DIM == 3 ? unfix24(b1[1]) : 0.0, Z = unfix24(b1[2]);
    int g[3] = {(int)(b1[0] >> 24), DIM == 3 ? (int)(b1[1] >> 24) : 0, (int)(b1[2] >> 24)};
    if (g[0] < 0 || g[0] >= S.n[0]) {
        X = wrap_periodic(X, S.nd[0]);
        g[0] += g[0] < 0 ? S.n[0] : -S.n[0];
    }
    if (DIM == 3 && (g[1] < 0 || g[1] >= S.n[1])) {
        Y = wrap_periodic(Y, S.nd[1]);
        g[1] += g[1] < 0 ? S.n[1] : -S.n[1];
    }
    int key = -1;
    if (S.absorb > 0) {
        if (g[2] < S.absorb || g[2] >= S.n[2] - S.absorb) key = S.ntiles;
    } else if (g[2] < 0 || g[2] >= S.n[2]) {
        Z = wrap_periodic(Z, S.nd[2]);
        g[2] += g[2] < 0 ? S.n[2] : -S.n[2];
    }
    if (key < 0) {
        bool own = (unsigned)(g[0] - tl.o[0]) < (unsigned)S.T[0] && (unsigned)(g[2] - tl.o[2]) < (unsigned)S.T[2];
        if (DIM == 3) own = own && (unsigned)(g[1] - tl.o[1]) < (unsigned)S.T[1];
        key = own ? tl.t
                  : tile_key(S, min(max(g[0], 0), S.n[0] - 1), DIM == 3 ? min(max(g[1], 0), S.n[1] - 1) : 0,
                             min(max(g[2], 0), S.n[2] - 1));
    }
    sp.cur[0][p] = X;
    if (DIM == 3) sp.cur[1][p] = Y;
    sp.cur[2][p] = Z;
    sp.cur[3][p] = f64_of(n0);
    sp.cur[4][p] = f64_of(n1);
    sp.cur[5][p] = f64_of(n2);
    sp.key[p] = key;
    warp_hist_add(sp.count, key);
}

// A warp deposits n <= 32 queued (cell-crossing) particles of its ring,
// starting at slot head, on the ORDER + 2 window: lane i takes entry head + i.
// Supports are taken relative to the origin of tile tl and the view V is that
// tile's; with the global J target any tile gives the same global nodes (the
// entries hold global positions), so rings then drain across tile changes.
template <class R, int DIM, int ORDER>
__device__ __forceinline__ void drain_warp(const SimDev& S, const Tile& tl,
                                           const JView& V,
                                           const double* __restrict__ sQw, unsigned head, unsigned n,
                                           const R* jf, int32_t* err) {
    using A = Arith<R>;
    const unsigned lane = threadIdx.x & 31u;
    if (lane >= n) return;
    const unsigned i = (head + lane) & (WQ - 1);
    const double X = sQw[0 * WQ + i], Z = sQw[1 * WQ + i];
    const double X1 = sQw[2 * WQ + i], Z1 = sQw[3 * WQ + i], qw = sQw[4 * WQ + i];
    const double Y = DIM == 3 ? sQw[5 * WQ + i] : 0.0, vy = DIM == 3 ? 0.0 : sQw[5 * WQ + i];
    const double Y1 = DIM == 3 ? sQw[6 * WQ + i] : 0.0;
    Support<ORDER, R> nd[3], mv[3];
    nd[0] = support_at<ORDER, R>(X, tl.o[0]);
    nd[2] = support_at<ORDER, R>(Z, tl.o[2]);
    mv[0] = support_at<ORDER, R>(X1, tl.o[0]);
    mv[2] = support_at<ORDER, R>(Z1, tl.o[2]);
    if (DIM == 3) {
        nd[1] = support_at<ORDER, R>(Y, tl.o[1]);
        mv[1] = support_at<ORDER, R>(Y1, tl.o[1]);
    } else {
        nd[1].s = -1;
        nd[1].w[0] = A::c(1.0);
        mv[1] = nd[1];
    }
    if (!deposit<R, DIM, ORDER, ORDER + 2>(S, V, A::from(qw), A::from(vy), jf, nd[0], nd[1], nd[2],
                                           mv[0], mv[1], mv[2]))
        atomicOr(err, PIC_DERR_BOUNDS);
}

// float-float keeps the drain out of line: the cell-crossing deposit is long
// and rare, and inlined into the particle loop it crowds the instruction cache
// (about 5 % of the kernel); FP64 is indifferent and inlines it, as does FP32
template <class R, int DIM, int ORDER>
__device__ __noinline__ void drain_warp_outlined(const SimDev& S, const Tile& tl,
                                                 const JView& V,
                                                 const double* __restrict__ sQw, unsigned head, unsigned n,
                                                 const R* jf, int32_t* err) {
    drain_warp<R, DIM, ORDER>(S, tl, V, sQw, head, n, jf, err);
}

template <class R, int DIM, int ORDER>
__device__ __forceinline__ void drain(const SimDev& S, const Tile& tl, const JView& V,
                                      const double* __restrict__ sQw, unsigned head, unsigned n,
                                      const R* jf, int32_t* err) {
    if constexpr (!std::is_same<R, dd>::value)
        drain_warp<R, DIM, ORDER>(S, tl, V, sQw, head, n, jf, err);
    else
        drain_warp_outlined<R, DIM, ORDER>(S, tl, V, sQw, head, n, jf, err);
}

// the J view of tile tl: the global padded arrays
__device__ __forceinline__ JView j_view(const SimDev& S, const Tile& tl) {
    JView v;
    const int lo = S.jlo;
    v.base = S.F[6] + pidx(S, tl.o[0] - lo, S.dim == 3 ? tl.o[1] - lo : 0, tl.o[2] - lo);
    v.cs = (int64_t)S.pn[0] * S.pn[1] * S.pn[2];
    v.sy = S.pn[0];
    v.sz = S.pn[0] * S.pn[1];
    return v;
}

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// the simulation's constants in the push arithmetic R
template <class R, int DIM>
struct SimConsts {
    R jf[3], dtd[3];
    __device__ __forceinline__ explicit SimConsts(const SimDev& S) {
        using A = Arith<R>;
        jf[0] = A::from(S.jfac[0]);
        jf[1] = A::from(DIM == 3 ? S.jfac[1] : S.jyfac2d);
        jf[2] = A::from(S.jfac[2]);
        dtd[0] = A::from(S.dtd[0]);
        dtd[1] = A::from(S.dtd[1]);
        dtd[2] = A::from(S.dtd[2]);
    }
};

// MINB = resident CTAs per SM the register allocation is sized for (1: up to
// 255 registers, 8 warps per SM; 2: at most 128 registers, 16 warps per SM).
// PREC = arithmetic of the particle push: 0 FP64, 1 float-float, 2 FP32 (storage,
// positions and index math stay FP64 in all three, and the current goes to the
// global FP64 J by L2 reductions).
// PPT = particles per thread per loop iteration: their HBM loads are issued
// together before the first of them is pushed (FP32 with PPT 1 stages each
// lane's next particle through shared memory instead).
template <int DIM, int ORDER, int MINB, int PREC, int PPT>
__global__ void __launch_bounds__(256, MINB) pic_particle_kernel(const SchedDev* __restrict__ sd,
                                                              SimDev* __restrict__ sims) {
    using R = typename std::conditional<PREC == 1, dd, typename std::conditional<PREC == 2, float, double>::type>::type;
    using A = Arith<R>;
    constexpr bool XD = PREC == 0 && ORDER == 1;  // x-difference tile beside the E/B tile
    constexpr bool FC = PREC == 2;                // E/B tile converted to floats in place; particle staging
    extern __shared__ __align__(128) double smem_raw[];
    __shared__ __align__(8) uint64_t bar;
    // TMA destinations must be 128-byte aligned: round the dynamic base up
    double* smem = reinterpret_cast<double*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~static_cast<uintptr_t>(127));
    __shared__ int s_unit, s_list, s_abort;
    __shared__ HotSim s_hot;
    __shared__ unsigned s_qhead[QMAXWARPS], s_qtail[QMAXWARPS];
    __shared__ unsigned long long s_cost;

    const int nlists = sd->meta[0];
    const int steal = sd->meta[1];
    const int my_list = blockIdx.x % nlists;
    if (threadIdx.x == 0) {
        mbar_init(&bar);
        s_list = my_list;
        s_abort = 0;
        for (int w = 0; w < QMAXWARPS; ++w) s_qhead[w] = s_qtail[w] = 0u;
        s_cost = 0ull;
    }
    __syncthreads();
    uint32_t phase = 0;
    Tile cur;
    cur.sim = -1;
    cur.t = -1;
    int visited = 0;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // ring of cell-crossing particles, in global scratch (L1/L2 resident; a
    // drain runs once per 32 crossings)
    double* const gring = sd->rings + ((size_t)blockIdx.x * QMAXWARPS + warp) * PIC_RING_DOUBLES;

    // a warp's ring of cell-crossing particles outlives tile changes (with the
    // global J every tile gives the same global nodes); it is drained when the
    // simulation changes (rings hold one simulation's particles, at that
    // simulation's queue offset) and at the end
    auto drain_ring = [&](const SimDev& CS) {
        const unsigned head = s_qhead[warp], tail = s_qtail[warp];
        if (tail != head) {
            const SimConsts<R, DIM> K(CS);
            drain<R, DIM, ORDER>(CS, cur, j_view(CS, cur), gring, head, tail - head, K.jf, sd->err);
            __syncwarp();
            if (lane == 0) s_qhead[warp] = tail;
            __syncwarp();
        }
    };

    while (true) {
        if (threadIdx.x == 0) {
            int u = -1;
            while (visited < nlists) {
                int L = s_list;
                int pos = atomicAdd(sd->head + L, 1);
                int b = sd->list_off[L], e = sd->list_off[L + 1];
                if (b + pos < e) { u = b + pos; break; }
                if (!steal) { visited = nlists; break; }
                s_list = (L + 1) % nlists;
                ++visited;
            }
            s_unit = u;
            // every warp has left the previous unit (its closing barrier): restage
            if (u >= 0) stage_hot(s_hot, sims[sd->units[u].sim]);
        }
        __syncthreads();
        const int u = s_unit;
        if (u < 0) break;
        const UnitDev unit = sd->units[u];
        const SimDev& S = sims[unit.sim];
        const bool cap_clk = (S.capture & 1) != 0, cap_time = (S.capture & 2) != 0;
        const uint64_t t_unit0 = (threadIdx.x == 0 && cap_time) ? globaltimer() : 0ull;
        const SmemPlan P = smem_plan(S.ebs, XD, FC);
        double* sEBd = smem;
        double* sDd = smem + 6 * P.eb_stride;   // x differences (linear FP64)
        const R* sEB = reinterpret_cast<const R*>(smem);
        unsigned long long my_clk = 0ull;
        const SimConsts<R, DIM> K(S);

        for (int spi = 0; spi < S.nsp; ++spi) {
            const SpeciesDev& sp = S.sp[spi];
            const R kq = A::from(sp.kq);
            const R qs = A::from(sp.q);
            const int t_first = unit.box * S.tiles_per_box;
            const int t_end = t_first + S.tiles_per_box;
            const int64_t b0 = sp.off[t_first], nbp = sp.off[t_end] - b0;
            const int64_t r0 = b0 + (nbp * unit.chunk) / unit.nchunks;
            const int64_t r1 = b0 + (nbp * (unit.chunk + 1)) / unit.nchunks;
            if (r0 >= r1) continue;
            for (int t = t_first; t < t_end; ++t) {
                const int64_t s0 = max(sp.off[t], r0), s1 = min(sp.off[t + 1], r1);
                if (s0 >= s1) continue;
                if (t != cur.t || unit.sim != cur.sim) {
                    if (cur.t >= 0 && unit.sim != cur.sim) drain_ring(sims[cur.sim]);
                    __syncthreads();
                    cur.sim = unit.sim;
                    cur.t = t;
                    tile_origin(S, t, cur.o);
                    if (threadIdx.x == 0) {
                        fence_proxy_async();
                        mbar_expect_tx(&bar, (uint32_t)(6 * P.eb_vol * sizeof(double)));
                        constexpr int H = EBHalo<ORDER>::lo;
                        const int x0 = cur.o[0] - H + S.g[0];
                        const int y0 = (DIM == 3) ? cur.o[1] - H + S.g[1] : 0;
                        const int z0 = cur.o[2] - H + S.g[2];
#pragma unroll
                        for (int c = 0; c < 6; ++c)
                            tma_load_3d(sEBd + c * P.eb_stride, &S.tmap[c], x0, y0, z0, &bar);
                    }
                    bool ok = mbar_wait_bounded(&bar, phase);
                    phase ^= 1u;
                    if (!ok) {
                        atomicOr(sd->err, PIC_DERR_TMA_TIMEOUT);
                        atomicExch(&s_abort, 1);
                    }
                    __syncthreads();
                    if (s_abort) {
                        // the copies may still be in flight: one more bounded wait, then leave
                        if (threadIdx.x == 0) mbar_wait_bounded(&bar, phase ^ 1u);
                        __syncthreads();
                        return;
                    }
                    if constexpr (XD) {
                        // x differences of every staged row (each x lerp of the gather
                        // becomes one FMA): one thread per row, walking along x
                        const int SX = S.ebs[0], rows = S.ebs[1] * S.ebs[2];
                        for (int i = threadIdx.x; i < 6 * rows; i += blockDim.x) {
                            const int c = i / rows, row = i - c * rows;
                            const double* f = sEBd + c * P.eb_stride + row * SX;
                            double* dst = sDd + c * P.d_stride + row * (SX - 1);
                            double prev = f[0];
                            for (int x = 1; x < SX; ++x) {
                                const double v = f[x];
                                dst[x - 1] = v - prev;
                                prev = v;
                            }
                        }
                        __syncthreads();
                    }
                    if constexpr (PREC == 1) {
                        // E/B tile to float pairs, in place (8 bytes either way)
                        for (int i = threadIdx.x; i < 6 * P.eb_stride; i += blockDim.x) {
                            const dd v = dd_from(sEBd[i]);
                            reinterpret_cast<dd*>(sEBd)[i] = v;
                        }
                        __syncthreads();
                    }
                    if constexpr (PREC == 2) {
                        // E/B tile to FP32 in place, in rounds of 8 elements per thread
                        // (nt threads); round m reads doubles [8 nt m, 8 nt (m + 1)] and,
                        // after its barrier, writes elements [8 nt m, 8 nt (m + 1)).
                        // Linear shapes: element i becomes the float pair (F[i],
                        // F[i+1] - F[i]) in the 8 bytes of double i (the pair at the end
                        // of a row is never read).  Other orders: element i becomes float
                        // i, overlaying doubles [4 nt m, 4 nt (m + 1)).  Either way a
                        // round writes only doubles read by rounds <= m and none read by a
                        // later round.
                        const int ntot = 6 * P.eb_stride, nt = blockDim.x;
                        for (int r0 = 0; r0 < ntot; r0 += 8 * nt) {
                            float v[8], d[8];
#pragma unroll
                            for (int k = 0; k < 8; ++k) {
                                const int i = r0 + k * nt + threadIdx.x;
                                v[k] = i < ntot ? f32_of(sEBd[i]) : 0.0f;
                                if constexpr (ORDER == 1) d[k] = i + 1 < ntot ? f32_of(sEBd[i + 1]) - v[k] : 0.0f;
                            }
                            __syncthreads();
#pragma unroll
                            for (int k = 0; k < 8; ++k) {
                                const int i = r0 + k * nt + threadIdx.x;
                                if (i < ntot) {
                                    if constexpr (ORDER == 1)
                                        reinterpret_cast<float2*>(sEBd)[i] = make_float2(v[k], d[k]);
                                    else
                                        reinterpret_cast<float*>(sEBd)[i] = v[k];
                                }
                            }
                        }
                        __syncthreads();
                    }
                }
                const unsigned long long c0 = cap_clk ? clock64() : 0ull;
                {
                    // per-warp loop: no CTA barrier until the tile changes
                    const JView V = j_view(S, cur);
                    double* sQw = gring;
                    const R* sD = XD ? reinterpret_cast<const R*>(sDd) : nullptr;
                    volatile unsigned* vtail = s_qtail + warp;
                    auto push = [&](int64_t p, const PIn& in) {
                        if constexpr (PREC == 2 && ORDER == 1)
                            push_one_f32lin<DIM>(s_hot, s_hot.sp[spi], cur, sEB, V, sQw, s_qtail + warp, P, K.jf,
                                                 K.dtd, kq, qs, p, in, sd->err);
                        else
                            push_one<R, DIM, ORDER>(s_hot, s_hot.sp[spi], cur, sEB, sD, V, sQw, s_qtail + warp, P,
                                                    K.jf, K.dtd, kq, qs, p, in, sd->err);
                    };
                    // a full ring (32 queued crossings) is drained by the whole warp
                    auto drain_full = [&]() {
                        __syncwarp();
                        const unsigned head = s_qhead[warp], tail = *vtail;
                        if (tail - head >= 32u) {
                            drain<R, DIM, ORDER>(S, cur, V, sQw, head, 32u, K.jf, sd->err);
                            __syncwarp();
                            if (lane == 0) s_qhead[warp] = head + 32u;
                            __syncwarp();
                        }
                    };
                    if constexpr (PREC == 2 && PPT == 1) {
                        // FP32: the particle loads are the latency the loop waits on; each
                        // lane stages its next particle into shared memory with cp.async
                        // one iteration ahead (two buffers per warp, the lane's own column)
                        double* const pbw = smem + P.pb_off + warp * (2 * PIN_SLOTS) + lane;
                        const int64_t pf = s0 + warp * 32 + lane;
                        if (pf < s1) stage_in<DIM>(s_hot.sp[spi], pf, pbw);
                        cp_async_commit();
                        unsigned buf = 0u;
                        for (int64_t p0 = s0 + warp * 32; p0 < s1; p0 += (int64_t)blockDim.x) {
                            const int64_t pn = p0 + blockDim.x + lane;
                            if (pn < s1) stage_in<DIM>(s_hot.sp[spi], pn, pbw + (buf ^ 1u) * PIN_SLOTS);
                            cp_async_commit();
                            cp_async_wait<1>();
                            const int64_t p = p0 + lane;
                            if (p < s1) push(p, read_staged<DIM>(pbw + buf * PIN_SLOTS));
                            buf ^= 1u;
                            drain_full();
                        }
                        cp_async_wait<0>();
                    } else {
                        for (int64_t p0 = s0 + warp * (32 * PPT); p0 < s1; p0 += (int64_t)blockDim.x * PPT) {
                            PIn in[PPT];
#pragma unroll
                            for (int q = 0; q < PPT; ++q) {
                                const int64_t p = p0 + q * 32 + lane;
                                if (p < s1) in[q] = load_one<DIM>(s_hot.sp[spi], p);
                            }
#pragma unroll
                            for (int q = 0; q < PPT; ++q) {
                                const int64_t p = p0 + q * 32 + lane;
                                if (p < s1) push(p, in[q]);
                                drain_full();
                            }
                        }
                    }
                    __syncwarp();
                }
                if (cap_clk) my_clk += clock64() - c0;
            }
        }
        // in-situ cost: thread clocks -> warp sum -> shared -> one global add per unit
        if (cap_clk) {
            unsigned long long ws = warp_sum_u64(my_clk);
            if ((threadIdx.x & 31) == 0 && ws) atomicAdd(&s_cost, ws);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            if (s_cost) atomicAdd((unsigned long long*)(S.cost_clock + unit.box), s_cost);
            s_cost = 0ull;
            // kernel-time cost: wall span of the unit on this CTA (ns)
            if (cap_time)
                atomicAdd((unsigned long long*)(S.cost_time + unit.box),
                          (unsigned long long)(globaltimer() - t_unit0));
        }
    }
    if (cur.t >= 0) drain_ring(sims[cur.sim]);
}

// ---- host side of one precision: launch, attributes, occupancy
template <int DIM, int ORDER, int PREC>
static cudaError_t launch_particles_t(const LaunchCfg& cfg, size_t smem, const SchedDev* sched,
                                      SimDev* sims, cudaStream_t st) {
    const bool two = cfg.ppt == 2;
    if (cfg.minb == 2) {
        if (two) pic_particle_kernel<DIM, ORDER, 2, PREC, 2><<<cfg.ctas, cfg.threads, smem, st>>>(sched, sims);
        else pic_particle_kernel<DIM, ORDER, 2, PREC, 1><<<cfg.ctas, cfg.threads, smem, st>>>(sched, sims);
    } else {
        if (two) pic_particle_kernel<DIM, ORDER, 1, PREC, 2><<<cfg.ctas, cfg.threads, smem, st>>>(sched, sims);
        else pic_particle_kernel<DIM, ORDER, 1, PREC, 1><<<cfg.ctas, cfg.threads, smem, st>>>(sched, sims);
    }
    return cudaGetLastError();
}

template <class K>
static cudaError_t set_smem(K kernel, size_t smem) {
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

template <int DIM, int ORDER, int PREC>
static cudaError_t prepare_t(size_t smem) {
    cudaError_t e = set_smem(pic_particle_kernel<DIM, ORDER, 1, PREC, 1>, smem);
    if (e == cudaSuccess) e = set_smem(pic_particle_kernel<DIM, ORDER, 2, PREC, 1>, smem);
    if (e == cudaSuccess) e = set_smem(pic_particle_kernel<DIM, ORDER, 1, PREC, 2>, smem);
    if (e == cudaSuccess) e = set_smem(pic_particle_kernel<DIM, ORDER, 2, PREC, 2>, smem);
    return e;
}

template <int DIM, int ORDER, int PREC>
static int occupancy_t(int minb, int ppt, int threads, size_t smem) {
    int n = 0;
    cudaError_t e;
    if (minb == 2)
        e = ppt == 2 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, pic_particle_kernel<DIM, ORDER, 2, PREC, 2>,
                                                                     threads, smem)
                     : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, pic_particle_kernel<DIM, ORDER, 2, PREC, 1>,
                                                                     threads, smem);
    else
        e = ppt == 2 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, pic_particle_kernel<DIM, ORDER, 1, PREC, 2>,
                                                                     threads, smem)
                     : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, pic_particle_kernel<DIM, ORDER, 1, PREC, 1>,
                                                                     threads, smem);
    return e == cudaSuccess ? n : 0;
}

// dispatch over the shape order for one precision (PIC_PREC) and one
// dimensionality (PIC_DIM): each translation unit instantiates one pair
#define PIC_DISPATCH_DO(FN, ...)                                            \
    do {                                                                    \
        if (order == 1) return FN<PIC_DIM, 1, PIC_PREC>(__VA_ARGS__);       \
        if (order == 2) return FN<PIC_DIM, 2, PIC_PREC>(__VA_ARGS__);       \
        if (order == 3) return FN<PIC_DIM, 3, PIC_PREC>(__VA_ARGS__);       \
    } while (0)

}  // namespace

// the three entry points of one translation unit, suffix SUF = p<prec>_d<dim>
#define PIC_DEFINE_PARTICLE_TU(SUF)                                                                      \
    cudaError_t pic_launch_particles_##SUF(int order, const LaunchCfg& cfg, size_t smem,                 \
                                           const SchedDev* sched, SimDev* sims, cudaStream_t st) {       \
        PIC_DISPATCH_DO(launch_particles_t, cfg, smem, sched, sims, st);                                  \
        return cudaErrorInvalidValue;                                                                     \
    }                                                                                                     \
    cudaError_t pic_prepare_particles_##SUF(int order, size_t smem) {                                     \
        PIC_DISPATCH_DO(prepare_t, smem);                                                                 \
        return cudaErrorInvalidValue;                                                                     \
    }                                                                                                     \
    int pic_particle_occupancy_##SUF(int order, int minb, int ppt, int threads, size_t smem) {            \
        PIC_DISPATCH_DO(occupancy_t, minb, ppt, threads, smem);                                           \
        return 0;                                                                                         \
    }
