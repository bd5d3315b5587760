// GB300 (sm_103a) kernels and C ABI of the thermal MRT lattice-Boltzmann
// hot path of arXiv:1809.08683 (declarations and conventions: include/lbm.h).
//
// Data layout in HBM, per lattice: two buffers (A, B), each 18 planes
// (f'_0..f'_8, g'_0..g'_8) of ny rows with a pitch of nx rounded up to 32
// elements, FP64 or FP32.  One time step is
//   fused kernel     : every node is loaded once from the current buffer,
//                      collided (Eqs. LBE.u.c, LBE.T.c) and pushed into the
//                      other buffer (Eqs. LBE.u.s, LBE.T.s); a population that
//                      would leave the domain is written back reversed into the
//                      node's own slot (Eqs. BB.f, BB.g);
//   k_boundary       : every wall node of the other buffer is rebuilt from its
//                      bounced sums, the wall data and the extrapolated
//                      redefined non-equilibrium moments (Sec. 3).
// The fused kernels sweep a run of rows of a strip of columns row by row:
// each row is staged into shared memory by one TMA tensor copy, and rho' and
// p' of the rows j-1, j, j+1 (plus one halo column on each side) stay in a
// shared-memory ring (block strips) or in registers and neighbouring lanes
// (warp strips), so the gradients of the correction terms T grad(rho) and
// X grad(p) need no extra pass over HBM.  The fused kernels are block strips
// (k_collide_stream), warp strips (k_collide_warp), paired block strips
// (k_collide_pair: two nodes per thread in packed FP32) and paired warp
// strips (k_collide_warp2); default_shape picks one per lattice and
// lbm_set_tile selects any other.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/lbm.h"
#include "lbm_f2.cuh"
#include "lbm_ff.cuh"
#include "lbm_node.cuh"

using lbm::f2;
using lbm::ff64;
using lbm::Mac;
using lbm::MacC;
using lbm::Params;

namespace {

// ------------------------------------------------------------------------
// device-side descriptors
// ------------------------------------------------------------------------

struct WallDev {
    double u[2];
    double T;
    int thermal;
    int order;
};

// Windows staged by one 3-D TMA copy per row: all 18 planes of a run of
// columns of one row of buffer b, described by tmap[k][b] over the tensor
// [18][ny][pitch].  k = 0: warp strips (kWinCols[0] columns); k = 1: paired
// warp strips (kWinCols[1], FP32 only); k = 2, 3, 4: block strips of 32, 64,
// 128 columns with a 16-byte chunk on either side.
constexpr int kWinCols[2] = {36, 68};
constexpr int kTmaps = 5;
__host__ __device__ constexpr int tmap_block_index(int bx) { return bx == 32 ? 2 : (bx == 64 ? 3 : 4); }

struct InstDesc {
    CUtensorMap tmap[kTmaps][2];  // first member: 64-byte aligned with the descriptor
    void* buf[2];
    long long plane;  // elements per plane
    int nx, ny, pitch, px, py;
    int precision;
    unsigned int* status;
    WallDev wall[4];
    Params<double> pd;
    Params<float> pf;
};

struct Work {  // one CTA of the fused kernel
    int inst, x0, y0, y1, par;
    int dir;          // block strips: 0 sweeps the run upwards (+y), 1 downwards
    long long step0;  // the lattice's step count when this table was built
};

struct BWork {  // one CTA of the wall pass
    int inst, k0, cnt, par;
};

template <typename R>
__device__ __forceinline__ const Params<R>& dparams(const InstDesc* D);
template <>
__device__ __forceinline__ const Params<double>& dparams<double>(const InstDesc* D) { return D->pd; }
template <>
__device__ __forceinline__ const Params<float>& dparams<float>(const InstDesc* D) { return D->pf; }


template <typename R>
__device__ __forceinline__ void load18(const R* __restrict__ base, long long plane, long long idx, R* v) {
#pragma unroll
    for (int q = 0; q < 18; ++q) v[q] = __ldg(base + q * plane + idx);
}

template <typename R>
__device__ __forceinline__ void store18(R* __restrict__ base, long long plane, long long idx, const R* v) {
#pragma unroll
    for (int q = 0; q < 18; ++q) base[q * plane + idx] = v[q];
}

template <int MC = lbm::MODEL_ANY, typename R>
__device__ __forceinline__ void node_macros(const Params<R>& P, const R* v, Mac<R>& m) {
    R rd, jx, jy, sg;
    lbm::node_sums(v, v + 9, rd, jx, jy, sg);
    lbm::macros<MC>(P, rd, jx, jy, sg, m);
}

template <typename R>
__device__ void load_params(Params<R>* dst, const Params<R>* src) {
    const int n = sizeof(Params<R>) / sizeof(int);
    const int* s = reinterpret_cast<const int*>(src);
    int* d = reinterpret_cast<int*>(dst);
    for (int i = threadIdx.x; i < n; i += blockDim.x) d[i] = s[i];
}

// Unbiased (stochastic) rounding of FP32 stores.  With round-to-nearest a
// nearly steady state repeats the same rounding error every step, which acts
// like a spurious body force of up to ulp(f')/2 per step; adding uniform noise
// of one ulp of the stored value before rounding makes the expected stored
// value equal the exact one.  The noise comes from a counter-based hash of
// (node, absolute step), so a lattice gives the same bits alone or batched.
__device__ __forceinline__ uint32_t mix32(uint32_t h) {
    h ^= h >> 16;
    h *= 0x7feb352du;
    h ^= h >> 15;
    h *= 0x846ca68bu;
    h ^= h >> 16;
    return h;
}

// One draw per node and step: the low 23 bits of the node's hash as the
// mantissa of a float in [1, 2), mapped to r * 2^-23 with r uniform in
// [-1/2, 1/2).  Multiplying by 2^e (a stored value with its mantissa
// cleared) gives r * ulp for normal values and 0 for zero.  Every stored
// value gets +r or -r (alternating over the links, opposite for f_i and
// g_i): each is rounded without bias, which is all the update needs; the
// 18 draws of a node are correlated, not independent.
__device__ __forceinline__ float dither_draw(uint32_t h) {
    return fmaf(__int_as_float(0x3f800000u | (h & 0x007fffffu)), 1.1920928955078125e-7f, -1.7881393432617188e-7f);
}
__device__ __forceinline__ float ulp_scale(float v) { return __int_as_float(__float_as_int(v) & 0x7f800000); }

struct AddDither {
    float r;
    mutable float s = 1.0f;  // sign of the next link's draw (folds to a constant once unrolled)
    __device__ __forceinline__ AddDither(uint32_t h, float scale) : r(dither_draw(h) * scale) {}
    __device__ __forceinline__ void operator()(float& f, float df, float& g, float dg) const {
        const float rs = s * r;
        f = f + fmaf(rs, ulp_scale(f), df);
        g = g + fmaf(-rs, ulp_scale(g), dg);
        s = -s;
    }
    __device__ __forceinline__ void operator()(double& f, double df, double& g, double dg) const {
        f = f + df;
        g = g + dg;
    }
};

// rho' and p' of node (xx, yy) read straight from a buffer.
template <int MC = lbm::MODEL_ANY, typename R>
__device__ void rho_p_at(const Params<R>& P, const R* __restrict__ src, long long plane, int pitch,
                         int xx, int yy, R& rd, R& pd) {
    R v[18];
    load18(src, plane, (long long)yy * pitch + xx, v);
    Mac<R> m;
    node_macros<MC>(P, v, m);
    rd = m.rho_d;
    pd = m.p_d;
}

// Push streaming of one node's post-collision DFs v[0..17] (f then g) from
// (x, j) into dst: population i moves to (x + e_ix, j + e_iy), wraps across
// a periodic edge, or, leaving the lattice through a wall, lands reversed in
// its own node's opposite slot (the bounce-back part of the wall treatment).
template <typename R>
__device__ __forceinline__ void push_node(R* __restrict__ dst, const R* v, int x, int j, int nx, int ny, int pitch,
                                          long long plane, int px, int py) {
    R* o = dst + ((long long)j * pitch + x);
    if (x >= 1 && x <= nx - 2 && j >= 1 && j <= ny - 2) {
        // interior: every population lands in the domain, no wrap;
        // 18 planes fit 32-bit offsets (checked at creation)
        const int pl = (int)plane;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const int ex = (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0);
            const int ey = (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
            const int off = ey * pitch + ex;
            o[i * pl + off] = v[i];
            o[(9 + i) * pl + off] = v[9 + i];
        }
    } else {
        // edge node: periodic wrap, or bounce-back into its own slot
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const int ex = (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0);
            const int ey = (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
            const int opp = (i == 0) ? 0 : (i <= 4 ? ((i + 1) & 3) + 1 : ((i - 3) & 3) + 5);
            int xd = x + ex, yd = j + ey;
            bool out = false;
            if (xd < 0 || xd >= nx) { if (px) xd = (xd < 0) ? nx - 1 : 0; else out = true; }
            if (yd < 0 || yd >= ny) { if (py) yd = (yd < 0) ? ny - 1 : 0; else out = true; }
            if (out) {
                o[opp * plane] = v[i];
                o[(9 + opp) * plane] = v[9 + i];
            } else {
                const long long t2 = (long long)yd * pitch + xd;
                dst[i * plane + t2] = v[i];
                dst[(9 + i) * plane + t2] = v[9 + i];
            }
        }
    }
}

// Push streaming of a pair of nodes (xa, j), (xa + 1, j) in packed FP32:
// populations that stream along y only land as one 8-byte store (xa is even
// and the pitch a multiple of 32); an edge pair goes node by node with
// periodic wrap or bounce-back.  act_b = false: only node xa exists.
__device__ __forceinline__ void push_pair(float* __restrict__ dst, const f2* v, int xa, bool act_b, int j, int nx, int ny,
                                          int pitch, long long plane, int px, int py) {
    const int xb = xa + 1;
    if (act_b && xa >= 1 && xb <= nx - 2 && j >= 1 && j <= ny - 2) {
        // both nodes interior: no wrap, no bounce-back
        float* o = dst + ((long long)j * pitch + xa);
        const int pl = (int)plane;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const int ex = (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0);
            const int ey = (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
            const int off = ey * pitch + ex;
            if (ex == 0) {
                *reinterpret_cast<float2*>(o + i * pl + off) = v[i].v;
                *reinterpret_cast<float2*>(o + (9 + i) * pl + off) = v[9 + i].v;
            } else {
                o[i * pl + off] = v[i].v.x;
                o[i * pl + off + 1] = v[i].v.y;
                o[(9 + i) * pl + off] = v[9 + i].v.x;
                o[(9 + i) * pl + off + 1] = v[9 + i].v.y;
            }
        }
    } else if (act_b && !px && j >= 1 && j <= ny - 2 && (xa == 0 || xb == nx - 1)) {
        // a pair holding one node of a walled x side, in a row away from the
        // y walls: the wall node's populations that would leave the lattice
        // land reversed in its own slots (Eqs. BB.f, BB.g), all others
        // stream as in the interior
        float* o = dst + ((long long)j * pitch + xa);
        const int pl = (int)plane;
        const bool west = xa == 0;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const int ex = (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0);
            const int ey = (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
            const int opp = (i == 0) ? 0 : (i <= 4 ? ((i + 1) & 3) + 1 : ((i - 3) & 3) + 5);
            const int off = ey * pitch + ex;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int q = h ? 9 + i : i, qo = h ? 9 + opp : opp;
                const float2 w = v[q].v;
                if (ex == 0) {
                    *reinterpret_cast<float2*>(o + q * pl + off) = w;
                } else if (west && ex < 0) {
                    o[qo * pl] = w.x;              // node a leaves through the west wall
                    o[q * pl + off + 1] = w.y;     // node b lands on column 0
                } else if (!west && ex > 0) {
                    o[q * pl + off] = w.x;         // node a lands on column nx - 1
                    o[qo * pl + 1] = w.y;          // node b leaves through the east wall
                } else {
                    o[q * pl + off] = w.x;
                    o[q * pl + off + 1] = w.y;
                }
            }
        }
    } else {
        // edge pair: per node, periodic wrap or bounce-back into its own slot
#pragma unroll
        for (int lane = 0; lane < 2; ++lane) {
            if (lane && !act_b) break;
            const int x = lane ? xb : xa;
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                const int ex = (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0);
                const int ey = (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
                const int opp = (i == 0) ? 0 : (i <= 4 ? ((i + 1) & 3) + 1 : ((i - 3) & 3) + 5);
                const float fv = lane ? v[i].v.y : v[i].v.x;
                const float gv = lane ? v[9 + i].v.y : v[9 + i].v.x;
                int xd = x + ex, yd = j + ey;
                bool out = false;
                if (xd < 0 || xd >= nx) { if (px) xd = (xd < 0) ? nx - 1 : 0; else out = true; }
                if (yd < 0 || yd >= ny) { if (py) yd = (yd < 0) ? ny - 1 : 0; else out = true; }
                if (out) {
                    const long long t2 = (long long)j * pitch + x;
                    dst[opp * plane + t2] = fv;
                    dst[(9 + opp) * plane + t2] = gv;
                } else {
                    const long long t2 = (long long)yd * pitch + xd;
                    dst[i * plane + t2] = fv;
                    dst[(9 + i) * plane + t2] = gv;
                }
            }
        }
    }
}

// ------------------------------------------------------------------------
// TMA bulk copies and mbarriers (inline PTX, sm_90+ forms valid on sm_103a)
// ------------------------------------------------------------------------

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: gives up after `limit` SM cycles, by default 2^32 (2 s at
// 2 GHz).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long limit = 1LL << 32) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > limit) return false;
    return true;
}

// Check of the timeout path: one thread waits, with the given limit, on an
// mbarrier that expects one arrival which nothing makes (no copy is issued),
// gives up and sets the same status bit as a fused kernel whose row copy
// never lands.
__global__ void k_wait_selftest(unsigned int* status, long long limit) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0 && !mbar_wait(&bar, 0, limit)) atomicOr(status, 2u);
}

// Global -> shared bulk copy completing on an mbarrier; addresses 16-byte
// aligned, size a multiple of 16 bytes.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

// Tensor copies need 128-byte aligned shared-memory destinations; a CTA
// whose dynamic shared memory is not aligned that way reports status bit 4
// and does nothing (the condition is the same for every thread of the CTA).
__device__ __forceinline__ bool smem_misaligned(const void* smem, unsigned int* status) {
    if ((smem_addr(smem) & 127u) == 0) return false;
    if (threadIdx.x == 0) atomicOr(status, 4u);
    return true;
}

// One 3-D tensor copy: the box of `tmap` at (x, y, z) into shared memory,
// completing on an mbarrier.  x * element size must be a multiple of 16
// bytes; the destination is 128-byte aligned; coordinates outside the
// tensor read as zero and still count towards the transaction bytes.
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* tmap, int x, int y, int z, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
            smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(tmap)), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
        : "memory");
}

// ------------------------------------------------------------------------
// fused collide + stream
// ------------------------------------------------------------------------

// rho' and p' of one node, adjacent so that the gradient stencil reads both
// with one shared-memory load.
template <typename R>
struct alignas(2 * sizeof(R)) RhoP {
    R r, p;
};

// Shared-memory layout of the block-strip kernel: S stages of one lattice
// row of the CTA's strip (18 planes, each [16-byte left-halo chunk][BX]
// [16-byte right-halo chunk], 128-byte aligned for the tensor copy), one
// mbarrier per stage, the parameters, and a 4-row ring of (rho', p') pairs
// over the strip plus its two halo columns.
template <typename R, int BX, int S>
struct FusedSmem {
    static constexpr int E = 16 / (int)sizeof(R);  // elements per 16-byte chunk
    static constexpr int W = BX + 2 * E;            // stage row width per plane
    static constexpr size_t stage_bytes = ((size_t)18 * W * sizeof(R) + 127) / 128 * 128;
    static constexpr size_t off_bars = (size_t)S * stage_bytes;
    static constexpr size_t off_params = off_bars + 8 * S;
    static constexpr size_t off_ring = (off_params + sizeof(Params<R>) + 15) / 16 * 16;
    static constexpr size_t bytes = off_ring + (size_t)2 * 4 * (BX + 2) * sizeof(R);
};

// Launch traits of the fused kernel: stage count (rows in flight = S - 2
// beyond the two being used) and the minimum resident CTAs per SM, which caps
// registers at 128 (FP32) or 255 (FP64) per thread.
template <typename R, int BX>
struct FusedTraits {
    static constexpr int S = BX == 32 ? 3 : 4;
    static constexpr int MINB = (sizeof(R) == 4 ? 512 : 256) / BX;
    static constexpr int MINB_LEAN = (sizeof(R) == 4 ? 640 : 256) / BX;  // about 100 registers in FP32
};

// KEEP = true carries each thread's macros from the row pass to the
// collision; KEEP = false recomputes them from the staged DFs, trading about
// 50 instructions per node for fewer registers and more resident warps.
template <typename R, int BX, int S, bool KEEP = true, int MC = lbm::MODEL_ANY>
__global__ void __launch_bounds__(BX, KEEP ? FusedTraits<R, BX>::MINB : FusedTraits<R, BX>::MINB_LEAN)
    k_collide_stream(const Work* __restrict__ work, InstDesc* const* __restrict__ descs, int step_par,
                     const long long* __restrict__ counter) {
    using L = FusedSmem<R, BX, S>;
    constexpr int E = L::E, W = L::W;
    constexpr size_t SST = L::stage_bytes / sizeof(R);  // elements from one stage to the next
    extern __shared__ __align__(128) unsigned char smem[];
    R* stage = reinterpret_cast<R*>(smem);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L::off_bars);
    Params<R>& P = *reinterpret_cast<Params<R>*>(smem + L::off_params);
    RhoP<R>(*s_rp)[BX + 2] = reinterpret_cast<RhoP<R>(*)[BX + 2]>(smem + L::off_ring);
    __shared__ int s_abort;

    const Work w = work[blockIdx.x];
    const InstDesc* D = descs[w.inst];
    if (smem_misaligned(smem, D->status)) return;
    load_params(&P, &dparams<R>(D));
    const int tid = threadIdx.x;
    if (tid == 0) {
        for (int k = 0; k < S; ++k) mbar_init(&bars[k], 1);
        fence_mbar_init();
        s_abort = 0;
    }
    const int nx = D->nx, ny = D->ny, pitch = D->pitch, px = D->px, py = D->py;
    const long long plane = D->plane;
    const int b = w.par ^ step_par;
    const R* __restrict__ src = reinterpret_cast<const R*>(D->buf[b]);
    R* __restrict__ dst = reinterpret_cast<R*>(D->buf[b ^ 1]);
    unsigned int* status = D->status;
    const uint32_t step_hash = mix32((uint32_t)(w.step0 + *counter) * 0x9e3779b1u + 0x632be5abu);
    __syncthreads();
    const float dscale = (float)P.dither;

    const int x = w.x0 + tid;
    const bool active = x < nx;
    const int xlast = min(w.x0 + BX, nx) - 1;
    const int tlast = xlast - w.x0;
    int xhl = w.x0 - 1;
    bool has_l = true;
    if (xhl < 0) { if (px) xhl = nx - 1; else has_l = false; }
    int xhr = xlast + 1;
    bool has_r = true;
    if (xhr >= nx) { if (px) xhr = 0; else has_r = false; }
    const int xcl = has_l ? (xhl / E) * E : 0, xcr = has_r ? (xhr / E) * E : 0;
    const int nmain = min(BX, pitch - w.x0);  // multiple of 32 elements: 16-byte sized
    const int nrows = w.y1 - w.y0;
    const int last_l = nrows + 1;             // logical rows 0..last_l = physical y0-1..y1 (dir 0)
    const int c = tid + 1;                    //                         or y1..y0-1 (dir 1)
    // Vertically adjacent runs sweep in opposite directions, so that the
    // rows they share (each one's halo rows) are read by both at about the
    // same time, the second time from L2.
    const bool down = w.dir != 0;

    // physical row of logical row l, or -1 if it lies outside a walled lattice
    auto phys = [&](int l) -> int {
        int y = down ? w.y1 - l : w.y0 - 1 + l;
        if (y < 0 || y >= ny) {
            if (!py) return -1;
            y = (y < 0) ? y + ny : y - ny;
        }
        return y;
    };

    // warp 0 issues the copies of logical row l into stage l % S; a row that
    // does not exist still completes its barrier phase (plain arrive)
    // a strip whose halo wraps across a periodic edge stages its row with
    // per-plane copies; any other with one tensor copy of columns
    // x0 - E .. x0 + BX + E - 1, which lays the stage out the same way
    const bool wraps = px && (w.x0 == 0 || xhr == 0);
    const CUtensorMap* tmap = &D->tmap[tmap_block_index(BX)][b];
    const uint32_t tx = wraps ? (uint32_t)(18 * (nmain * (int)sizeof(R) + 16 * (has_l + has_r)))
                              : (uint32_t)(18 * W * (int)sizeof(R));
    int issued = 0, waited = 0;  // logical rows issued / waited for by this thread
    auto issue = [&](int l) {
        if (l > last_l || tid >= 32) return;
        issued = l + 1;
        const int s = l % S;
        const int y = phys(l);
        if (tid == 0) {
            if (y < 0) mbar_arrive(&bars[s]);
            else mbar_arrive_expect_tx(&bars[s], tx);
        }
        __syncwarp();
        if (y >= 0 && !wraps) {
            if (tid == 0) {
                fence_proxy_async();
                tma_load_3d(stage + (size_t)s * SST, tmap, w.x0 - E, y, 0, &bars[s]);
            }
        } else if (y >= 0 && tid < 18) {
            fence_proxy_async();
            const R* row = src + tid * plane + (long long)y * pitch;
            R* st = stage + (size_t)s * SST + (size_t)tid * W;
            bulk_g2s(st + E, row + w.x0, (uint32_t)(nmain * sizeof(R)), &bars[s]);
            if (has_l) bulk_g2s(st, row + xcl, 16u, &bars[s]);
            if (has_r) bulk_g2s(st + E + BX, row + xcr, 16u, &bars[s]);
        }
    };

    // wait for logical row l and put its rho', p' into ring slot l % 4;
    // active threads also return their own node's macros in m
    auto row_macros = [&](int l, MacC<R>& mk) -> bool {
        const int s = l % S;
        if (!mbar_wait(&bars[s], (uint32_t)((l / S) & 1))) {
            atomicOr(status, 2u);
            s_abort = 1;
            return false;
        }
        waited = l + 1;
        const R* st = stage + (size_t)s * SST;
        const int slot = l & 3;
        if (active) {
            R v[18];
#pragma unroll
            for (int q = 0; q < 18; ++q) v[q] = st[q * W + E + tid];
            Mac<R> m;
            node_macros<MC>(P, v, m);
            compress(m, mk);
            s_rp[slot][c] = RhoP<R>{m.rho_d, m.p_d};
        }
        // the two halo columns: two adjacent lanes of one warp run the same
        // instruction stream on their own chunk, in warp 1 (not the warp
        // that issues the copies) when the strip has more than one warp
        constexpr int HL = BX >= 64 ? 32 : 0;
        const bool hl = (tid == HL && has_l), hr = (tid == HL + 1 && has_r);
        if (hl || hr) {
            const int off = hl ? (xhl - xcl) : (E + BX + (xhr - xcr));
            const int col = hl ? 0 : tlast + 2;
            R v[18];
#pragma unroll
            for (int q = 0; q < 18; ++q) v[q] = st[q * W + off];
            Mac<R> h;
            node_macros<MC>(P, v, h);
            s_rp[slot][col] = RhoP<R>{h.rho_d, h.p_d};
        }
        return true;
    };

    for (int l = 0; l < S; ++l) issue(l);
    MacC<R> mc, mn;
    if (phys(0) >= 0) row_macros(0, mn);
    row_macros(1, mc);

    for (int k = 0; k < nrows; ++k) {
        const int j = down ? w.y1 - 1 - k : w.y0 + k;
        if (phys(k + 2) >= 0) row_macros(k + 2, mn);
        __syncthreads();
        if (s_abort) break;
        issue(k + S);  // stage of logical row k is free: its collision finished before the barrier

        if (active) {
            if (KEEP && !(isfinite(mc.rho_d) && isfinite(mc.T_d))) atomicOr(status, 1u);
            // ring slots of the rows j - 1 (sm), j, j + 1 (sp)
            const int sm = (down ? k + 2 : k) & 3, s0 = (k + 1) & 3, sp = (down ? k : k + 2) & 3;
            const bool onS = !py && j == 0, onN = !py && j == ny - 1;
            const bool onW = !px && x == 0, onE = !px && x == nx - 1;
            R grx, gry, gpx, gpy;
            if (!(onS || onN || onW || onE)) {
                // grad = 3 sum_i w_i e_i phi(x + e_i), w = 1/9 (axis), 1/36 (diagonal)
                const R t = R(1.0 / 3.0), d = R(1.0 / 12.0);
                const RhoP<R> ml = s_rp[sm][c - 1], mc_ = s_rp[sm][c], mr = s_rp[sm][c + 1];
                const RhoP<R> zl = s_rp[s0][c - 1], zr = s_rp[s0][c + 1];
                const RhoP<R> pl = s_rp[sp][c - 1], pc = s_rp[sp][c], pr = s_rp[sp][c + 1];
                grx = t * (zr.r - zl.r) + d * ((pr.r - pl.r) + (mr.r - ml.r));
                gry = t * (pc.r - mc_.r) + d * ((pr.r - mr.r) + (pl.r - ml.r));
                gpx = t * (zr.p - zl.p) + d * ((pr.p - pl.p) + (mr.p - ml.p));
                gpy = t * (pc.p - mc_.p) + d * ((pr.p - mr.p) + (pl.p - ml.p));
            } else {
                // wall node: one-sided second order along the inward normal,
                // central along the wall
                const R r0 = s_rp[s0][c].r, p0 = s_rp[s0][c].p;
                if (onW || onE) {
                    const int dx = onW ? 1 : -1;
                    R r2, p2;
                    rho_p_at<MC>(P, src, plane, pitch, x + 2 * dx, j, r2, p2);
                    const R r1 = s_rp[s0][c + dx].r, p1 = s_rp[s0][c + dx].p;
                    grx = R(dx) * (R(-3) * r0 + R(4) * r1 - r2) * R(0.5);
                    gpx = R(dx) * (R(-3) * p0 + R(4) * p1 - p2) * R(0.5);
                } else {
                    grx = (s_rp[s0][c + 1].r - s_rp[s0][c - 1].r) * R(0.5);
                    gpx = (s_rp[s0][c + 1].p - s_rp[s0][c - 1].p) * R(0.5);
                }
                if (onS || onN) {
                    const int dy = onS ? 1 : -1;
                    R r2, p2;
                    rho_p_at<MC>(P, src, plane, pitch, x, j + 2 * dy, r2, p2);
                    const R r1 = onS ? s_rp[sp][c].r : s_rp[sm][c].r;
                    const R p1 = onS ? s_rp[sp][c].p : s_rp[sm][c].p;
                    gry = R(dy) * (R(-3) * r0 + R(4) * r1 - r2) * R(0.5);
                    gpy = R(dy) * (R(-3) * p0 + R(4) * p1 - p2) * R(0.5);
                } else {
                    gry = (s_rp[sp][c].r - s_rp[sm][c].r) * R(0.5);
                    gpy = (s_rp[sp][c].p - s_rp[sm][c].p) * R(0.5);
                }
            }

            R v[18];
            const R* st = stage + (size_t)((k + 1) % S) * SST + E + tid;
#pragma unroll
            for (int q = 0; q < 18; ++q) v[q] = st[q * W];
            Mac<R> mf;
            if (KEEP) {
                lbm::expand<MC>(P, mc, mf);
            } else {
                node_macros<MC>(P, v, mf);
                if (!(isfinite(mf.rho_d) && isfinite(mf.T_d))) atomicOr(status, 1u);
            }
            AddDither add(mix32(step_hash ^ ((uint32_t)j * 0x85ebca77u + (uint32_t)x * 0xc2b2ae3du)), dscale);
            // block strips keep the DFs in registers through the collision
            // (no spills at 128 registers; re-reading them cost 0.6%)
            lbm::collide<MC>(P, mf, v, v + 9, grx, gry, gpx, gpy, add);

            push_node(dst, v, x, j, nx, ny, pitch, plane, px, py);
        }
        if (KEEP) mc = mn;
    }
    if (s_abort && tid == 0) {
        // leave no bulk copy in flight into this CTA's shared memory: wait,
        // in order, for every row issued and not yet waited for
        for (int l = waited; l < issued; ++l)
            if (phys(l) >= 0) mbar_wait(&bars[l % S], (uint32_t)((l / S) & 1));
    }
}

// ------------------------------------------------------------------------
// fused collide + stream, one autonomous warp per strip
// ------------------------------------------------------------------------

// Columns owned by one warp of k_collide_warp: lanes 1..30 own columns
// wx0 .. wx0 + 29; lane 0 holds column wx0 - 1 and lane 31 column wx0 + 30,
// whose macros the gradient stencil needs.
constexpr int kWarpCols = 30;

// Shared-memory layout of k_collide_warp: per warp, S stages of one lattice
// row and S mbarriers; then the parameters.  A stage holds the window
// [18 planes][MW columns] that one tensor copy writes, then, for a periodic
// edge, [18 planes][left wrap chunk, right wrap chunk].  The window starts at
// the 16-byte boundary at or below column wx0 - 1 and covers up to column
// wx0 + 30.
template <typename R, int NW, int S>
struct WarpSmem {
    static constexpr int E = 16 / (int)sizeof(R);  // elements per 16-byte chunk
    static constexpr int MW = kWinCols[0];
    static constexpr size_t wrap_off = (size_t)18 * MW * sizeof(R);  // bytes
    static constexpr size_t stage_bytes = (wrap_off + (size_t)18 * 2 * E * sizeof(R) + 127) / 128 * 128;
    static constexpr size_t warp_bytes = (size_t)S * stage_bytes;
    static constexpr size_t off_bars = (size_t)NW * warp_bytes;
    static constexpr size_t off_params = (off_bars + 8 * NW * S + 15) / 16 * 16;
    static constexpr size_t bytes = off_params + sizeof(Params<R>);
};

template <typename R>
struct WarpTraits {
    static constexpr int S = 3;
    static constexpr int WARPS_PER_SM = sizeof(R) == 4 ? 16 : 8;  // caps registers at 128 (FP32) / 255 (FP64)
};

// Same per-node arithmetic as k_collide_stream, bit for bit, with no
// block-wide synchronisation: each warp of the CTA sweeps its own strip of
// kWarpCols columns over the CTA's rows, stages rows by TMA into its own
// ring of stages, and takes the macros of the neighbouring columns from the
// neighbouring lanes (warp shuffles) and those of the rows j - 1, j, j + 1
// from its own registers.  Warps of a CTA only share the parameters.
template <typename R, int NW, int S, int MC = lbm::MODEL_ANY>
__global__ void __launch_bounds__(32 * NW, WarpTraits<R>::WARPS_PER_SM / NW)
    k_collide_warp(const Work* __restrict__ work, InstDesc* const* __restrict__ descs, int step_par,
                   const long long* __restrict__ counter) {
    using L = WarpSmem<R, NW, S>;
    constexpr int E = L::E, MW = L::MW;
    constexpr unsigned FULL = 0xffffffffu;
    extern __shared__ __align__(128) unsigned char smem[];
    Params<R>& P = *reinterpret_cast<Params<R>*>(smem + L::off_params);

    const Work w = work[blockIdx.x];
    const InstDesc* D = descs[w.inst];
    if (smem_misaligned(smem, D->status)) return;
    load_params(&P, &dparams<R>(D));
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned char* wstage = smem + (size_t)wid * L::warp_bytes;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L::off_bars) + wid * S;
    if (lane == 0) {
        for (int k = 0; k < S; ++k) mbar_init(&bars[k], 1);
        fence_mbar_init();
    }
    const int nx = D->nx, ny = D->ny, pitch = D->pitch, px = D->px, py = D->py;
    const long long plane = D->plane;
    const int b = w.par ^ step_par;
    const R* __restrict__ src = reinterpret_cast<const R*>(D->buf[b]);
    R* __restrict__ dst = reinterpret_cast<R*>(D->buf[b ^ 1]);
    unsigned int* status = D->status;
    const uint32_t step_hash = mix32((uint32_t)(w.step0 + *counter) * 0x9e3779b1u + 0x632be5abu);
    __syncthreads();  // parameters and barrier initialisation visible; the last block-wide barrier
    const float dscale = (float)P.dither;

    const int wx0 = w.x0 + kWarpCols * wid;
    if (wx0 >= nx) return;  // whole warp beyond a ragged right edge
    const int x = wx0 + lane - 1;  // this lane's column
    const bool owned = lane >= 1 && lane <= kWarpCols && x < nx;
    const int a = (max(wx0 - 1, 0) / E) * E;  // window start (16-byte aligned)
    const bool wrap_l = px && wx0 == 0;                 // lane 0 holds column nx - 1
    const bool wrap_r = px && wx0 + kWarpCols >= nx;    // lane nx - wx0 + 1 holds column 0
    const int cl = ((nx - 1) / E) * E;
    // the lane's column: window column `off`, or (wrapped) element `off` of
    // the wrap chunks; off < 0: no column
    int off = -1;
    const bool in_wrap = (x == -1 && wrap_l) || (x == nx && wrap_r);
    if (x >= 0 && x < nx) off = x - a;
    else if (x == -1 && wrap_l) off = nx - 1 - cl;
    else if (x == nx && wrap_r) off = E;
    const CUtensorMap* tmap = &D->tmap[0][b];
    const uint32_t tx = (uint32_t)(18 * (MW + (wrap_l ? E : 0) + (wrap_r ? E : 0)) * (int)sizeof(R));
    const int nrows = w.y1 - w.y0;
    const int last_l = nrows + 1;  // logical rows 0..last_l = physical y0-1..y1

    auto phys = [&](int l) -> int {
        int y = w.y0 - 1 + l;
        if (y < 0 || y >= ny) {
            if (!py) return -1;
            y = (y < 0) ? y + ny : y - ny;
        }
        return y;
    };

    // the warp issues the copies of logical row l into its stage l % S; a row
    // that does not exist still completes its barrier phase (plain arrive)
    int issued = 0;  // logical rows whose copies this warp has issued
    auto issue = [&](int l) {
        if (l > last_l) return;
        issued = l + 1;
        const int s = l % S;
        const int y = phys(l);
        if (lane == 0) {
            if (y < 0) mbar_arrive(&bars[s]);
            else mbar_arrive_expect_tx(&bars[s], tx);
        }
        __syncwarp();
        if (y >= 0) {
            unsigned char* st = wstage + (size_t)s * L::stage_bytes;
            if (lane == 0) {
                fence_proxy_async();
                tma_load_3d(st, tmap, a, y, 0, &bars[s]);
            }
            if ((wrap_l || wrap_r) && lane < 18) {
                fence_proxy_async();
                const R* row = src + lane * plane + (long long)y * pitch;
                R* wb = reinterpret_cast<R*>(st + L::wrap_off) + 2 * E * lane;
                if (wrap_l) bulk_g2s(wb, row + cl, 16u, &bars[s]);
                if (wrap_r) bulk_g2s(wb + E, row, 16u, &bars[s]);
            }
        }
    };

    // this lane's 18 DFs from stage s
    auto load_node = [&](int s, R* v) {
        const unsigned char* st = wstage + (size_t)s * L::stage_bytes;
        if (!in_wrap) {
            const R* p = reinterpret_cast<const R*>(st) + off;
#pragma unroll
            for (int q = 0; q < 18; ++q) v[q] = p[q * MW];
        } else {
            const R* p = reinterpret_cast<const R*>(st + L::wrap_off) + off;
#pragma unroll
            for (int q = 0; q < 18; ++q) v[q] = p[q * 2 * E];
        }
    };

    // wait for logical row l; lanes holding a column return its macros
    auto row_macros = [&](int l, MacC<R>& mk, R& r, R& p) -> bool {
        const int s = l % S;
        const bool ok = __all_sync(FULL, mbar_wait(&bars[s], (uint32_t)((l / S) & 1)));
        if (ok && off >= 0) {
            R v[18];
            load_node(s, v);
            Mac<R> m;
            node_macros<MC>(P, v, m);
            compress(m, mk);
            r = m.rho_d;
            p = m.p_d;
        } else {
            r = R(0);
            p = R(0);
        }
        return ok;
    };

    for (int l = 0; l < S; ++l) issue(l);
    int waited = 0;  // logical rows whose copies this warp has waited for
    MacC<R> mc, mn;
    R rm = R(0), pm = R(0), r0 = R(0), p0 = R(0), rp = R(0), pp = R(0);
    bool ok = true;
    if (phys(0) >= 0) ok = row_macros(0, mn, rm, pm);
    if (ok) {
        waited = 1;
        ok = row_macros(1, mc, r0, p0);
    }
    if (ok) waited = 2;

    for (int k = 0; ok && k < nrows; ++k) {
        const int j = w.y0 + k;
        if (phys(k + 2) >= 0) ok = row_macros(k + 2, mn, rp, pp);
        if (!ok) break;
        waited = k + 3;
        issue(k + S);  // stage of logical row k is free: the warp's last collision read it

        const R rml = __shfl_up_sync(FULL, rm, 1), rmr = __shfl_down_sync(FULL, rm, 1);
        const R r0l = __shfl_up_sync(FULL, r0, 1), r0r = __shfl_down_sync(FULL, r0, 1);
        const R rpl = __shfl_up_sync(FULL, rp, 1), rpr = __shfl_down_sync(FULL, rp, 1);
        const R pml = __shfl_up_sync(FULL, pm, 1), pmr = __shfl_down_sync(FULL, pm, 1);
        const R p0l = __shfl_up_sync(FULL, p0, 1), p0r = __shfl_down_sync(FULL, p0, 1);
        const R ppl = __shfl_up_sync(FULL, pp, 1), ppr = __shfl_down_sync(FULL, pp, 1);
        if (owned) {
            if (!(isfinite(mc.rho_d) && isfinite(mc.T_d))) atomicOr(status, 1u);
            const bool onS = !py && j == 0, onN = !py && j == ny - 1;
            const bool onW = !px && x == 0, onE = !px && x == nx - 1;
            R grx, gry, gpx, gpy;
            if (!(onS || onN || onW || onE)) {
                // grad = 3 sum_i w_i e_i phi(x + e_i), w = 1/9 (axis), 1/36 (diagonal)
                const R t = R(1.0 / 3.0), d = R(1.0 / 12.0);
                grx = t * (r0r - r0l) + d * ((rpr - rpl) + (rmr - rml));
                gry = t * (rp - rm) + d * ((rpr - rmr) + (rpl - rml));
                gpx = t * (p0r - p0l) + d * ((ppr - ppl) + (pmr - pml));
                gpy = t * (pp - pm) + d * ((ppr - pmr) + (ppl - pml));
            } else {
                // wall node: one-sided second order along the inward normal,
                // central along the wall
                if (onW || onE) {
                    const int dx = onW ? 1 : -1;
                    R r2, p2;
                    rho_p_at<MC>(P, src, plane, pitch, x + 2 * dx, j, r2, p2);
                    const R r1 = onW ? r0r : r0l, p1 = onW ? p0r : p0l;
                    grx = R(dx) * (R(-3) * r0 + R(4) * r1 - r2) * R(0.5);
                    gpx = R(dx) * (R(-3) * p0 + R(4) * p1 - p2) * R(0.5);
                } else {
                    grx = (r0r - r0l) * R(0.5);
                    gpx = (p0r - p0l) * R(0.5);
                }
                if (onS || onN) {
                    const int dy = onS ? 1 : -1;
                    R r2, p2;
                    rho_p_at<MC>(P, src, plane, pitch, x, j + 2 * dy, r2, p2);
                    const R r1 = onS ? rp : rm, p1 = onS ? pp : pm;
                    gry = R(dy) * (R(-3) * r0 + R(4) * r1 - r2) * R(0.5);
                    gpy = R(dy) * (R(-3) * p0 + R(4) * p1 - p2) * R(0.5);
                } else {
                    gry = (rp - rm) * R(0.5);
                    gpy = (pp - pm) * R(0.5);
                }
            }

            R v[18];
            const int sc = (k + 1) % S;
            load_node(sc, v);
            Mac<R> mf;
            lbm::expand<MC>(P, mc, mf);
            AddDither add(mix32(step_hash ^ ((uint32_t)j * 0x85ebca77u + (uint32_t)x * 0xc2b2ae3du)), dscale);
            // the DFs are fetched again for the final update, so that they
            // need not occupy registers through the collision
            auto reload = [&](R* f, R*) {
                asm volatile("" ::: "memory");
                load_node(sc, f);  // f and g are v and v + 9: all 18 DFs
            };
            lbm::collide<MC>(P, mf, v, v + 9, grx, gry, gpx, gpy, add, reload);
            push_node(dst, v, x, j, nx, ny, pitch, plane, px, py);
        }
        mc = mn;
        rm = r0; pm = p0;
        r0 = rp; p0 = pp;
    }
    if (!ok) {
        atomicOr(status, 2u);
        // leave no bulk copy in flight into this warp's stages: wait, in
        // order, for every row issued and not yet waited for
        if (lane == 0)
            for (int l = waited; l < issued; ++l)
                if (phys(l) >= 0) mbar_wait(&bars[l % S], (uint32_t)((l / S) & 1));
        __syncwarp();
    }
}

// ------------------------------------------------------------------------
// fused collide + stream, two nodes per thread in packed FP32
// ------------------------------------------------------------------------

// Packed-pair variant of the FP32 fused kernel: thread t owns the columns
// x0 + 2t and x0 + 2t + 1 of its strip and evaluates the node arithmetic
// once for both, in packed FP32 (lbm_f2.cuh).  Row staging, the macro ring and
// the push are those of k_collide_stream; shared-memory loads are 8-byte
// pairs, and populations that stream along y only are stored as pairs.
template <int BX>
struct PairSmem {
    static constexpr int S = 3;
    static constexpr int E = 4;              // floats per 16-byte halo chunk
    static constexpr int W = BX + 2 * E;
    static constexpr int RW = BX + 4;        // ring row: x - x0 + 2, halos at 1 and (xlast - x0) + 3
    static constexpr size_t stage_bytes = ((size_t)18 * W * sizeof(float) + 127) / 128 * 128;
    static constexpr size_t off_bars = (size_t)S * stage_bytes;
    static constexpr size_t off_p2 = (off_bars + 8 * S + 15) / 16 * 16;
    static constexpr size_t off_p1 = (off_p2 + sizeof(Params<f2>) + 15) / 16 * 16;
    static constexpr size_t off_ring = (off_p1 + sizeof(Params<float>) + 15) / 16 * 16;
    static constexpr size_t bytes = off_ring + (size_t)2 * 4 * RW * sizeof(float);
};

__device__ void broadcast_params(const Params<float>& a, Params<f2>& b) {
#define BP(f) b.f = f2(a.f)
    BP(rho0); BP(T0); BP(E0); BP(Cv); BP(inv_Cv); BP(Rg); BP(eos_a); BP(eos_b); BP(p0); BP(rho0E0_p0);
    BP(rho0Cp0); BP(mu0); BP(inv_T0); BP(visc_S); BP(lam_fac); BP(tj_fac); BP(e_fac); BP(alpha1);
    BP(beta1); BP(alpha2); BP(beta2); BP(kk); BP(hh); BP(bb); BP(gamma1); BP(gamma2); BP(cR11);
    BP(cR17); BP(cR18); BP(cR71); BP(cR77); BP(cR81); BP(cR88); BP(Fx); BP(Fy); BP(cs_b0); BP(dither);
#undef BP
    b.eos = a.eos;
    b.visc = a.visc;
    b.force_mode = a.force_mode;
    b.corrections = a.corrections;
}

// Stochastic rounding of a pair of nodes: one draw per node and link.
// The rounding of AddDither for a pair of nodes: one draw per node, from
// the pair's hash and from its Weyl successor.
struct AddDither2 {
    float2 r;
    mutable float s = 1.0f;
    __device__ __forceinline__ AddDither2(uint32_t h, float scale)
        : r(make_float2(dither_draw(h) * scale, dither_draw(h + 0x9e3779b9u) * scale)) {}
    __device__ __forceinline__ void operator()(f2& f, f2 df, f2& g, f2 dg) const {
        const float2 rs = make_float2(s * r.x, s * r.y), rn = make_float2(-rs.x, -rs.y);
        f = f2(__fadd2_rn(f.v, __ffma2_rn(rs, make_float2(ulp_scale(f.v.x), ulp_scale(f.v.y)), df.v)));
        g = f2(__fadd2_rn(g.v, __ffma2_rn(rn, make_float2(ulp_scale(g.v.x), ulp_scale(g.v.y)), dg.v)));
        s = -s;
    }
};

#ifndef LBM_PAIR_WARPS_PER_SM
#define LBM_PAIR_WARPS_PER_SM 12  // resident warps per SM with the row macros kept in registers
#endif

template <int BX, bool KEEP, int MC = lbm::MODEL_ANY>
__global__ void __launch_bounds__(BX / 2, (KEEP ? LBM_PAIR_WARPS_PER_SM : 12) * 64 / BX) k_collide_pair(const Work* __restrict__ work,
                                                                    InstDesc* const* __restrict__ descs,
                                                                    int step_par, const long long* __restrict__ counter) {
    using L = PairSmem<BX>;
    constexpr int E = L::E, W = L::W, S = L::S, RW = L::RW;
    constexpr size_t SST = L::stage_bytes / sizeof(float);  // floats from one stage to the next
    extern __shared__ __align__(128) unsigned char smem[];
    float* stage = reinterpret_cast<float*>(smem);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L::off_bars);
    Params<f2>& P2 = *reinterpret_cast<Params<f2>*>(smem + L::off_p2);
    Params<float>& P1 = *reinterpret_cast<Params<float>*>(smem + L::off_p1);
    float(*s_rho)[RW] = reinterpret_cast<float(*)[RW]>(smem + L::off_ring);
    float(*s_p)[RW] = s_rho + 4;
    __shared__ int s_abort;

    const Work w = work[blockIdx.x];
    const InstDesc* D = descs[w.inst];
    if (smem_misaligned(smem, D->status)) return;
    load_params(&P1, &D->pf);
    const int tid = threadIdx.x;
    if (tid == 0) {
        for (int k = 0; k < S; ++k) mbar_init(&bars[k], 1);
        fence_mbar_init();
        s_abort = 0;
    }
    const int nx = D->nx, ny = D->ny, pitch = D->pitch, px = D->px, py = D->py;
    const long long plane = D->plane;
    const int b = w.par ^ step_par;
    const float* __restrict__ src = reinterpret_cast<const float*>(D->buf[b]);
    float* __restrict__ dst = reinterpret_cast<float*>(D->buf[b ^ 1]);
    unsigned int* status = D->status;
    const uint32_t step_hash = mix32((uint32_t)(w.step0 + *counter) * 0x9e3779b1u + 0x632be5abu);
    __syncthreads();
    if (tid == 0) broadcast_params(P1, P2);
    __syncthreads();
    const float dscale = P1.dither;

    const int xa = w.x0 + 2 * tid, xb = xa + 1;
    const bool act_a = xa < nx, act_b = xb < nx;
    const int xlast = min(w.x0 + BX, nx) - 1;
    int xhl = w.x0 - 1;
    bool has_l = true;
    if (xhl < 0) { if (px) xhl = nx - 1; else has_l = false; }
    int xhr = xlast + 1;
    bool has_r = true;
    if (xhr >= nx) { if (px) xhr = 0; else has_r = false; }
    const int xcl = has_l ? (xhl / E) * E : 0, xcr = has_r ? (xhr / E) * E : 0;
    const int nmain = min(BX, pitch - w.x0);
    const int nrows = w.y1 - w.y0;
    const int last_l = nrows + 1;
    const int ca = 2 * tid + 2;                 // ring column of x_a
    const int cr = (xlast - w.x0) + 3;          // ring column of the right halo
    // vertically adjacent runs sweep in opposite directions (as in
    // k_collide_stream): logical rows 0..last_l are physical y0-1..y1 or y1..y0-1
    const bool down = w.dir != 0;

    auto phys = [&](int l) -> int {
        int y = down ? w.y1 - l : w.y0 - 1 + l;
        if (y < 0 || y >= ny) {
            if (!py) return -1;
            y = (y < 0) ? y + ny : y - ny;
        }
        return y;
    };

    // one tensor copy per row unless the halo wraps across a periodic edge
    // (a window of more than 256 columns takes per-plane copies too)
    constexpr bool kTensor = BX + 2 * E <= 256;
    const bool wraps = !kTensor || (px && (w.x0 == 0 || xhr == 0));
    const CUtensorMap* tmap = &D->tmap[tmap_block_index(kTensor ? BX : 128)][b];
    const uint32_t tx = wraps ? (uint32_t)(18 * (nmain * 4 + 16 * (has_l + has_r))) : (uint32_t)(18 * W * 4);
    int issued = 0, waited = 0;  // logical rows issued / waited for by this thread
    auto issue = [&](int l) {
        if (l > last_l || tid >= 32) return;
        issued = l + 1;
        const int s = l % S;
        const int y = phys(l);
        if (tid == 0) {
            if (y < 0) mbar_arrive(&bars[s]);
            else mbar_arrive_expect_tx(&bars[s], tx);
        }
        __syncwarp();
        if (y >= 0 && !wraps) {
            if (tid == 0) {
                fence_proxy_async();
                tma_load_3d(stage + (size_t)s * SST, tmap, w.x0 - E, y, 0, &bars[s]);
            }
        } else if (y >= 0 && tid < 18) {
            fence_proxy_async();
            const float* row = src + tid * plane + (long long)y * pitch;
            float* st = stage + (size_t)s * SST + (size_t)tid * W;
            bulk_g2s(st + E, row + w.x0, (uint32_t)(nmain * 4), &bars[s]);
            if (has_l) bulk_g2s(st, row + xcl, 16u, &bars[s]);
            if (has_r) bulk_g2s(st + E + BX, row + xcr, 16u, &bars[s]);
        }
    };

    auto row_macros = [&](int l, MacC<f2>& mk) -> bool {
        const int s = l % S;
        if (!mbar_wait(&bars[s], (uint32_t)((l / S) & 1))) {
            atomicOr(status, 2u);
            s_abort = 1;
            return false;
        }
        waited = l + 1;
        const float* st = stage + (size_t)s * SST;
        const int slot = l & 3;
        if (act_a) {
            f2 v[18];
#pragma unroll
            for (int q = 0; q < 18; ++q) v[q] = f2(*reinterpret_cast<const float2*>(st + q * W + E + 2 * tid));
            f2 rd, jx, jy, sg;
            lbm::node_sums(v, v + 9, rd, jx, jy, sg);
            Mac<f2> m;
            lbm::macros<MC>(P2, rd, jx, jy, sg, m);
            compress(m, mk);
            if (act_b) {
                *reinterpret_cast<float2*>(&s_rho[slot][ca]) = m.rho_d.v;
                *reinterpret_cast<float2*>(&s_p[slot][ca]) = m.p_d.v;
            } else {
                // a half-filled last pair: its second column is the right
                // halo, which another lane writes
                s_rho[slot][ca] = m.rho_d.v.x;
                s_p[slot][ca] = m.p_d.v.x;
            }
        }
        // halo columns in scalar arithmetic, on two adjacent lanes of one
        // warp (warp 1 when there are two or more), after their own pairs
        constexpr int HL = BX / 2 >= 64 ? 32 : 0;
        const bool hl = (tid == HL && has_l), hr = (tid == HL + 1 && has_r);
        if (hl || hr) {
            const int off = hl ? (xhl - xcl) : (E + BX + (xhr - xcr));
            const int col = hl ? 1 : cr;
            float v[18];
            Mac<float> h;
#pragma unroll
            for (int q = 0; q < 18; ++q) v[q] = st[q * W + off];
            node_macros<MC>(P1, v, h);
            s_rho[slot][col] = h.rho_d;
            s_p[slot][col] = h.p_d;
        }
        return true;
    };

    for (int l = 0; l < S; ++l) issue(l);
    MacC<f2> mc, mn;
    if (phys(0) >= 0) row_macros(0, mn);
    row_macros(1, mc);

    for (int k = 0; k < nrows; ++k) {
        const int j = down ? w.y1 - 1 - k : w.y0 + k;
        if (phys(k + 2) >= 0) row_macros(k + 2, mn);
        __syncthreads();
        if (s_abort) break;
        issue(k + S);

        if (act_a) {
            if (KEEP && !(isfinite(mc.rho_d.v.x) && isfinite(mc.T_d.v.x) && isfinite(mc.rho_d.v.y) && isfinite(mc.T_d.v.y)))
                atomicOr(status, act_b ? 1u : ((isfinite(mc.rho_d.v.x) && isfinite(mc.T_d.v.x)) ? 0u : 1u));
            // ring slots of the rows j - 1 (sm), j, j + 1 (sp)
            const int sm = (down ? k + 2 : k) & 3, s0 = (k + 1) & 3, sp = (down ? k : k + 2) & 3;
            // interior stencil for both nodes: columns (ca-1, ca) on the left, (ca+1, ca+2) on the right
            auto grad = [&](float (*a)[RW], f2& gx, f2& gy) {
                const float2 cm = *reinterpret_cast<const float2*>(&a[sm][ca]);
                const float2 c0 = *reinterpret_cast<const float2*>(&a[s0][ca]);
                const float2 cp = *reinterpret_cast<const float2*>(&a[sp][ca]);
                const f2 lm(make_float2(a[sm][ca - 1], cm.x)), rm(make_float2(cm.y, a[sm][ca + 2]));
                const f2 l0(make_float2(a[s0][ca - 1], c0.x)), r0(make_float2(c0.y, a[s0][ca + 2]));
                const f2 lp(make_float2(a[sp][ca - 1], cp.x)), rp(make_float2(cp.y, a[sp][ca + 2]));
                const f2 t(1.0f / 3.0f), d(1.0f / 12.0f);
                gx = t * (r0 - l0) + d * ((rp - lp) + (rm - lm));
                gy = t * (f2(cp) - f2(cm)) + d * ((rp - rm) + (lp - lm));
            };
            f2 grx, gry, gpx, gpy;
            grad(s_rho, grx, gry);
            grad(s_p, gpx, gpy);
            const bool rowwall = !py && (j == 0 || j == ny - 1);
            const bool colwall = !px && (xa == 0 || xb >= nx - 1);
            if (rowwall || colwall) {
                // wall nodes: one-sided second order along the inward normal,
                // central along the wall (scalar, per node of the pair)
#pragma unroll
                for (int lane = 0; lane < 2; ++lane) {
                    const int x = lane ? xb : xa;
                    if (lane && !act_b) break;
                    const int c = ca + lane;
                    const bool onS = !py && j == 0, onN = !py && j == ny - 1;
                    const bool onW = !px && x == 0, onE = !px && x == nx - 1;
                    if (!(onS || onN || onW || onE)) continue;
                    // rho', p' two nodes inward: along x from the ring when the
                    // strip or one of its halo columns holds that column, else
                    // (and along y) from the source buffer
                    const int dx = onW ? 1 : -1, dy = onS ? 1 : -1;
                    float rx2 = 0.0f, px2 = 0.0f, ry2 = 0.0f, py2 = 0.0f;
                    if (onW || onE) {
                        const int c2 = c + 2 * dx;
                        if ((c2 >= 2 && c2 < cr) || (c2 == 1 && has_l) || (c2 == cr && has_r)) {
                            rx2 = s_rho[s0][c2];
                            px2 = s_p[s0][c2];
                        } else {
                            rho_p_at<MC>(P1, src, plane, pitch, x + 2 * dx, j, rx2, px2);
                        }
                    }
                    if (onS || onN) rho_p_at<MC>(P1, src, plane, pitch, x, j + 2 * dy, ry2, py2);
                    float gr[4];
#pragma unroll
                    for (int fld = 0; fld < 2; ++fld) {
                        float (*a)[RW] = fld ? s_p : s_rho;
                        const float v0 = a[s0][c];
                        float gxs, gys;
                        if (onW || onE) {
                            gxs = (float)dx * (-3.0f * v0 + 4.0f * a[s0][c + dx] - (fld ? px2 : rx2)) * 0.5f;
                        } else {
                            gxs = (a[s0][c + 1] - a[s0][c - 1]) * 0.5f;
                        }
                        if (onS || onN) {
                            const float v1 = onS ? a[sp][c] : a[sm][c];
                            gys = (float)dy * (-3.0f * v0 + 4.0f * v1 - (fld ? py2 : ry2)) * 0.5f;
                        } else {
                            gys = (a[sp][c] - a[sm][c]) * 0.5f;
                        }
                        gr[2 * fld] = gxs;
                        gr[2 * fld + 1] = gys;
                    }
                    if (lane) { grx.v.y = gr[0]; gry.v.y = gr[1]; gpx.v.y = gr[2]; gpy.v.y = gr[3]; }
                    else { grx.v.x = gr[0]; gry.v.x = gr[1]; gpx.v.x = gr[2]; gpy.v.x = gr[3]; }
                }
            }

            f2 v[18];
            const float* st = stage + (size_t)((k + 1) % S) * SST + E + 2 * tid;
#pragma unroll
            for (int q = 0; q < 18; ++q) v[q] = f2(*reinterpret_cast<const float2*>(st + q * W));
            Mac<f2> mf;
            if (KEEP) {
                lbm::expand<MC>(P2, mc, mf);
            } else {
                f2 rd, jx, jy, sg;
                lbm::node_sums(v, v + 9, rd, jx, jy, sg);
                lbm::macros<MC>(P2, rd, jx, jy, sg, mf);
                if (!(isfinite(mf.rho_d.v.x) && isfinite(mf.T_d.v.x) && (!act_b || (isfinite(mf.rho_d.v.y) && isfinite(mf.T_d.v.y)))))
                    atomicOr(status, 1u);
            }
            AddDither2 add(mix32(step_hash ^ ((uint32_t)j * 0x85ebca77u + (uint32_t)xa * 0xc2b2ae3du)), dscale);
            auto reload = [&](f2* f, f2* g) {
                asm volatile("" ::: "memory");
#pragma unroll
                for (int q = 0; q < 9; ++q) {
                    f[q] = f2(*reinterpret_cast<const float2*>(st + q * W));
                    g[q] = f2(*reinterpret_cast<const float2*>(st + (9 + q) * W));
                }
            };
            lbm::collide<MC>(P2, mf, v, v + 9, grx, gry, gpx, gpy, add, reload);

            push_pair(dst, v, xa, act_b, j, nx, ny, pitch, plane, px, py);
        }
        if (KEEP) mc = mn;
    }
    if (s_abort && tid == 0) {
        // wait, in order, for every row issued and not yet waited for
        for (int l = waited; l < issued; ++l)
            if (phys(l) >= 0) mbar_wait(&bars[l % S], (uint32_t)((l / S) & 1));
    }
}

// ------------------------------------------------------------------------
// fused collide + stream, one autonomous warp per strip, two nodes per lane
// ------------------------------------------------------------------------

// Columns owned by one warp of k_collide_warp2: lane L = 1..30 owns the
// columns wx0 + 2L - 2 and wx0 + 2L - 1; lane 0 holds column wx0 - 1 (its
// second element) and lane 31 column wx0 + 60 (its first element).
constexpr int kWarp2Cols = 60;

// Stage layout as in WarpSmem, with a window of columns floor4(wx0 - 2) ..
// floor4(wx0 - 2) + 67.
template <int NW, int S>
struct Warp2Smem {
    static constexpr int E = 4;  // floats per 16-byte chunk
    static constexpr int MW = kWinCols[1];
    static constexpr size_t wrap_off = (size_t)18 * MW * sizeof(float);
    static constexpr size_t stage_bytes = (wrap_off + (size_t)18 * 2 * E * sizeof(float) + 127) / 128 * 128;
    static constexpr size_t warp_bytes = (size_t)S * stage_bytes;
    static constexpr size_t off_bars = (size_t)NW * warp_bytes;
    static constexpr size_t off_p2 = (off_bars + 8 * NW * S + 15) / 16 * 16;
    static constexpr size_t off_p1 = (off_p2 + sizeof(Params<f2>) + 15) / 16 * 16;
    static constexpr size_t bytes = off_p1 + sizeof(Params<float>);
};

// The warp-strip scheme of k_collide_warp with the node arithmetic of
// k_collide_pair: each lane evaluates two neighbouring nodes at once in
// packed FP32 (lbm_f2.cuh), including the macros of the strip's halo
// columns.  Neighbour macros come from the lane itself (the other node of
// its pair) or from the adjacent lane by shuffle.
#ifndef LBM_WARP2_WARPS_PER_SM
#define LBM_WARP2_WARPS_PER_SM 12  // resident warps per SM: 168 registers per thread
#endif

template <int NW, int S>
__global__ void __launch_bounds__(32 * NW, LBM_WARP2_WARPS_PER_SM / NW)
    k_collide_warp2(const Work* __restrict__ work, InstDesc* const* __restrict__ descs, int step_par,
                    const long long* __restrict__ counter) {
    using L = Warp2Smem<NW, S>;
    constexpr int E = L::E, MW = L::MW;
    constexpr unsigned FULL = 0xffffffffu;
    extern __shared__ __align__(128) unsigned char smem[];
    Params<f2>& P2 = *reinterpret_cast<Params<f2>*>(smem + L::off_p2);
    Params<float>& P1 = *reinterpret_cast<Params<float>*>(smem + L::off_p1);

    const Work w = work[blockIdx.x];
    const InstDesc* D = descs[w.inst];
    if (smem_misaligned(smem, D->status)) return;
    load_params(&P1, &D->pf);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned char* wstage = smem + (size_t)wid * L::warp_bytes;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L::off_bars) + wid * S;
    if (lane == 0) {
        for (int k = 0; k < S; ++k) mbar_init(&bars[k], 1);
        fence_mbar_init();
    }
    const int nx = D->nx, ny = D->ny, pitch = D->pitch, px = D->px, py = D->py;
    const long long plane = D->plane;
    const int b = w.par ^ step_par;
    const float* __restrict__ src = reinterpret_cast<const float*>(D->buf[b]);
    float* __restrict__ dst = reinterpret_cast<float*>(D->buf[b ^ 1]);
    unsigned int* status = D->status;
    const uint32_t step_hash = mix32((uint32_t)(w.step0 + *counter) * 0x9e3779b1u + 0x632be5abu);
    __syncthreads();
    if (threadIdx.x == 0) broadcast_params(P1, P2);
    __syncthreads();  // the last block-wide barrier
    const float dscale = P1.dither;

    const int wx0 = w.x0 + kWarp2Cols * wid;
    if (wx0 >= nx) return;
    const int xa = wx0 + 2 * lane - 2, xb = xa + 1;
    const bool own = lane >= 1 && lane <= kWarp2Cols / 2;
    const bool act_a = own && xa < nx, act_b = own && xb < nx;
    const int a0 = (max(wx0 - 2, 0) / E) * E;
    const bool wrap_l = px && wx0 == 0;
    const bool wrap_r = px && wx0 + kWarp2Cols >= nx;
    const int cl = ((nx - 1) / E) * E;
    // where column x sits as seen from this warp: window column o (o < MW),
    // element o - MW of the wrap chunks (o >= MW), or -1 if not held
    auto offset_of = [&](int x) -> int {
        if (x >= 0 && x < nx && x >= a0 && x - a0 < MW) return x - a0;
        if (x == -1 && wrap_l) return MW + (nx - 1 - cl);
        if (x == nx && wrap_r) return MW + E;
        return -1;
    };
    const int offa = offset_of(xa), offb = offset_of(xb);
    // both nodes in the window (offa is even): one 8-byte load per plane
    const bool fast = offa >= 0 && offa < MW && offb == offa + 1;
    const CUtensorMap* tmap = &D->tmap[1][b];
    const uint32_t tx = (uint32_t)(18 * (MW + (wrap_l ? E : 0) + (wrap_r ? E : 0)) * (int)sizeof(float));
    const int nrows = w.y1 - w.y0;
    const int last_l = nrows + 1;

    auto phys = [&](int l) -> int {
        int y = w.y0 - 1 + l;
        if (y < 0 || y >= ny) {
            if (!py) return -1;
            y = (y < 0) ? y + ny : y - ny;
        }
        return y;
    };

    int issued = 0;
    auto issue = [&](int l) {
        if (l > last_l) return;
        issued = l + 1;
        const int s = l % S;
        const int y = phys(l);
        if (lane == 0) {
            if (y < 0) mbar_arrive(&bars[s]);
            else mbar_arrive_expect_tx(&bars[s], tx);
        }
        __syncwarp();
        if (y >= 0) {
            unsigned char* st = wstage + (size_t)s * L::stage_bytes;
            if (lane == 0) {
                fence_proxy_async();
                tma_load_3d(st, tmap, a0, y, 0, &bars[s]);
            }
            if ((wrap_l || wrap_r) && lane < 18) {
                fence_proxy_async();
                const float* row = src + lane * plane + (long long)y * pitch;
                float* wb = reinterpret_cast<float*>(st + L::wrap_off) + 2 * E * lane;
                if (wrap_l) bulk_g2s(wb, row + cl, 16u, &bars[s]);
                if (wrap_r) bulk_g2s(wb + E, row, 16u, &bars[s]);
            }
        }
    };

    // the lane's two nodes from stage s (a column not held reads as 0)
    auto load_pair = [&](int s, f2* v) {
        const float* st = reinterpret_cast<const float*>(wstage + (size_t)s * L::stage_bytes);
        if (fast) {
#pragma unroll
            for (int q = 0; q < 18; ++q) v[q] = f2(*reinterpret_cast<const float2*>(st + q * MW + offa));
        } else {
            const float* wr = reinterpret_cast<const float*>(wstage + (size_t)s * L::stage_bytes + L::wrap_off);
            auto elem = [&](int o, int q) -> float {
                if (o < 0) return 0.0f;
                return o < MW ? st[q * MW + o] : wr[q * 2 * E + (o - MW)];
            };
#pragma unroll
            for (int q = 0; q < 18; ++q) v[q] = f2(make_float2(elem(offa, q), elem(offb, q)));
        }
    };

    auto row_macros = [&](int l, MacC<f2>& mk, f2& r, f2& p) -> bool {
        const int s = l % S;
        const bool ok = __all_sync(FULL, mbar_wait(&bars[s], (uint32_t)((l / S) & 1)));
        if (ok && (offa >= 0 || offb >= 0)) {
            f2 v[18];
            load_pair(s, v);
            f2 rd, jx, jy, sg;
            lbm::node_sums(v, v + 9, rd, jx, jy, sg);
            Mac<f2> m;
            lbm::macros(P2, rd, jx, jy, sg, m);
            compress(m, mk);
            r = m.rho_d;
            p = m.p_d;
        } else {
            r = f2(0.0f);
            p = f2(0.0f);
        }
        return ok;
    };

    for (int l = 0; l < S; ++l) issue(l);
    int waited = 0;
    MacC<f2> mc, mn;
    f2 rm(0.0f), pm(0.0f), r0(0.0f), p0(0.0f), rp(0.0f), pp(0.0f);
    bool ok = true;
    if (phys(0) >= 0) ok = row_macros(0, mn, rm, pm);
    if (ok) {
        waited = 1;
        ok = row_macros(1, mc, r0, p0);
    }
    if (ok) waited = 2;

    for (int k = 0; ok && k < nrows; ++k) {
        const int j = w.y0 + k;
        if (phys(k + 2) >= 0) ok = row_macros(k + 2, mn, rp, pp);
        if (!ok) break;
        waited = k + 3;
        issue(k + S);

        // left neighbour of node a: the previous lane's node b; right
        // neighbour of node b: the next lane's node a
        const float rmL = __shfl_up_sync(FULL, rm.v.y, 1), rmR = __shfl_down_sync(FULL, rm.v.x, 1);
        const float r0L = __shfl_up_sync(FULL, r0.v.y, 1), r0R = __shfl_down_sync(FULL, r0.v.x, 1);
        const float rpL = __shfl_up_sync(FULL, rp.v.y, 1), rpR = __shfl_down_sync(FULL, rp.v.x, 1);
        const float pmL = __shfl_up_sync(FULL, pm.v.y, 1), pmR = __shfl_down_sync(FULL, pm.v.x, 1);
        const float p0L = __shfl_up_sync(FULL, p0.v.y, 1), p0R = __shfl_down_sync(FULL, p0.v.x, 1);
        const float ppL = __shfl_up_sync(FULL, pp.v.y, 1), ppR = __shfl_down_sync(FULL, pp.v.x, 1);
        if (act_a) {
            if (!(isfinite(mc.rho_d.v.x) && isfinite(mc.T_d.v.x)) ||
                (act_b && !(isfinite(mc.rho_d.v.y) && isfinite(mc.T_d.v.y))))
                atomicOr(status, 1u);
            // the stencil for both nodes: left columns (xa - 1, xa), right (xb, xb + 1)
            auto grad = [&](const f2& cm, const f2& c0, const f2& cp, float mL, float mR, float zL, float zR, float pL,
                            float pR, f2& gx, f2& gy) {
                const f2 lm(make_float2(mL, cm.v.x)), rmv(make_float2(cm.v.y, mR));
                const f2 l0(make_float2(zL, c0.v.x)), r0v(make_float2(c0.v.y, zR));
                const f2 lp(make_float2(pL, cp.v.x)), rpv(make_float2(cp.v.y, pR));
                const f2 t(1.0f / 3.0f), d(1.0f / 12.0f);
                gx = t * (r0v - l0) + d * ((rpv - lp) + (rmv - lm));
                gy = t * (cp - cm) + d * ((rpv - rmv) + (lp - lm));
            };
            f2 grx, gry, gpx, gpy;
            grad(rm, r0, rp, rmL, rmR, r0L, r0R, rpL, rpR, grx, gry);
            grad(pm, p0, pp, pmL, pmR, p0L, p0R, ppL, ppR, gpx, gpy);
            const bool rowwall = !py && (j == 0 || j == ny - 1);
            const bool colwall = !px && (xa == 0 || xb >= nx - 1);
            if (rowwall || colwall) {
                // wall nodes: one-sided second order along the inward normal,
                // central along the wall (scalar, per node of the pair)
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const int x = e ? xb : xa;
                    if (e && !act_b) break;
                    const bool onS = !py && j == 0, onN = !py && j == ny - 1;
                    const bool onW = !px && x == 0, onE = !px && x == nx - 1;
                    if (!(onS || onN || onW || onE)) continue;
                    float gr[4];
#pragma unroll
                    for (int fld = 0; fld < 2; ++fld) {
                        const f2& c0f = fld ? p0 : r0;
                        const f2& cmf = fld ? pm : rm;
                        const f2& cpf = fld ? pp : rp;
                        const float v0 = e ? c0f.v.y : c0f.v.x;
                        // row-j values of the left and right neighbours of this node
                        const float left = e ? c0f.v.x : (fld ? p0L : r0L);
                        const float right = e ? (fld ? p0R : r0R) : c0f.v.y;
                        float gxs, gys;
                        if (onW || onE) {
                            const int dx = onW ? 1 : -1;
                            float r2, p2;
                            rho_p_at(P1, src, plane, pitch, x + 2 * dx, j, r2, p2);
                            gxs = (float)dx * (-3.0f * v0 + 4.0f * (onW ? right : left) - (fld ? p2 : r2)) * 0.5f;
                        } else {
                            gxs = (right - left) * 0.5f;
                        }
                        const float vm = e ? cmf.v.y : cmf.v.x, vp = e ? cpf.v.y : cpf.v.x;
                        if (onS || onN) {
                            const int dy = onS ? 1 : -1;
                            float r2, p2;
                            rho_p_at(P1, src, plane, pitch, x, j + 2 * dy, r2, p2);
                            const float v1 = onS ? vp : vm;
                            gys = (float)dy * (-3.0f * v0 + 4.0f * v1 - (fld ? p2 : r2)) * 0.5f;
                        } else {
                            gys = (vp - vm) * 0.5f;
                        }
                        gr[2 * fld] = gxs;
                        gr[2 * fld + 1] = gys;
                    }
                    if (e) { grx.v.y = gr[0]; gry.v.y = gr[1]; gpx.v.y = gr[2]; gpy.v.y = gr[3]; }
                    else { grx.v.x = gr[0]; gry.v.x = gr[1]; gpx.v.x = gr[2]; gpy.v.x = gr[3]; }
                }
            }

            f2 v[18];
            load_pair((k + 1) % S, v);
            Mac<f2> mf;
            expand(P2, mc, mf);
            AddDither2 add(mix32(step_hash ^ ((uint32_t)j * 0x85ebca77u + (uint32_t)xa * 0xc2b2ae3du)), dscale);
            auto reload = [&](f2* f, f2*) {
                asm volatile("" ::: "memory");
                load_pair((k + 1) % S, f);  // f and g are v and v + 9: all 18 DFs
            };
            lbm::collide(P2, mf, v, v + 9, grx, gry, gpx, gpy, add, reload);
            push_pair(dst, v, xa, act_b, j, nx, ny, pitch, plane, px, py);
        }
        mc = mn;
        rm = r0; pm = p0;
        r0 = rp; p0 = pp;
    }
    if (!ok) {
        atomicOr(status, 2u);
        if (lane == 0)
            for (int l = waited; l < issued; ++l)
                if (phys(l) >= 0) mbar_wait(&bars[l % S], (uint32_t)((l / S) & 1));
        __syncwarp();
    }
}

// ------------------------------------------------------------------------
// wall pass (Sec. 3)
// ------------------------------------------------------------------------

struct WallNode {
    int x, y, dx, dy;  // position and inward normal
    double ux, uy, T;
    int thermal, order;
};

__device__ __host__ inline int wall_count(int nx, int ny, int px, int py) {
    if (px && py) return 0;
    if (!py && px) return 2 * nx;
    if (py && !px) return 2 * ny;
    return 2 * nx + 2 * (ny - 2);
}

// k-th wall node: south row, north row, then west and east columns
// (without the corners when the rows exist).
__device__ void wall_node(const InstDesc* D, int k, WallNode& n) {
    const int nx = D->nx, ny = D->ny, px = D->px, py = D->py;
    int x, y;
    if (!py) {
        if (k < nx) { x = k; y = 0; }
        else if (k < 2 * nx) { x = k - nx; y = ny - 1; }
        else {
            int r = k - 2 * nx;
            if (r < ny - 2) { x = 0; y = r + 1; }
            else { x = nx - 1; y = r - (ny - 2) + 1; }
        }
    } else {
        if (k < ny) { x = 0; y = k; }
        else { x = nx - 1; y = k - ny; }
    }
    const bool onS = !py && y == 0, onN = !py && y == ny - 1;
    const bool onW = !px && x == 0, onE = !px && x == nx - 1;
    n.x = x;
    n.y = y;
    n.dx = onW ? 1 : (onE ? -1 : 0);
    n.dy = onS ? 1 : (onN ? -1 : 0);
    const WallDev* ws = onS ? &D->wall[0] : (onN ? &D->wall[1] : nullptr);
    const WallDev* wx = onW ? &D->wall[2] : (onE ? &D->wall[3] : nullptr);
    if (ws && wx) {
        // corner: at rest, x-side order, Dirichlet wins (x-side first)
        n.ux = 0.0;
        n.uy = 0.0;
        n.order = wx->order;
        if (wx->thermal == 0) { n.thermal = 0; n.T = wx->T; }
        else if (ws->thermal == 0) { n.thermal = 0; n.T = ws->T; }
        else { n.thermal = 1; n.T = 0.0; }
    } else {
        const WallDev* ww = ws ? ws : wx;
        n.ux = ww->u[0];
        n.uy = ww->u[1];
        n.thermal = ww->thermal;
        n.T = ww->T;
        n.order = ww->order;
    }
}

// Resident CTAs per SM of the FP32 wall pass.  3 leaves 146 registers per
// thread and no spills; 4 spilled 68 bytes per thread and took 0.1055 ms per
// step of the 96-cavity batch against 0.098 ms (6 and 8 CTAs, with more
// spills: 0.137 and 0.159 ms).  The pass is latency-bound, and the spill
// traffic costs more than the extra warps hide.
#ifndef LBM_BOUNDARY_MINB
#define LBM_BOUNDARY_MINB 3
#endif
template <typename R>
__global__ void __launch_bounds__(128, sizeof(R) == 4 ? LBM_BOUNDARY_MINB : 2) k_boundary(const BWork* __restrict__ work,
                                                  InstDesc* const* __restrict__ descs, int step_par,
                                                  long long* __restrict__ counter) {
    __shared__ Params<R> P;
    // the last wall-pass launch of a step advances the step counter that the
    // next step's fused launch reads
    if (counter && blockIdx.x == 0 && threadIdx.x == 0) *counter += 1;
    const BWork w = work[blockIdx.x];
    if (w.cnt <= 0) return;
    const InstDesc* D = descs[w.inst];
    load_params(&P, &dparams<R>(D));
    __syncthreads();
    if ((int)threadIdx.x >= w.cnt) return;
    const int k = w.k0 + threadIdx.x;
    const int pitch = D->pitch;
    const long long plane = D->plane;
    R* __restrict__ buf = reinterpret_cast<R*>(D->buf[(w.par ^ step_par) ^ 1]);
    WallNode n;
    wall_node(D, k, n);

    // the wall node's and x_f's populations, loaded together so that their
    // latencies overlap (the pass is bound by them).  On a walled x side away
    // from the corners the two nodes are neighbours in one row: when the
    // pair starts on an even column it comes as one 8-byte (FP32) or
    // 16-byte (FP64) load per population, which halves the load
    // instructions and the DRAM sectors touched of a column of wall nodes.
    R v[18], u[18];
    const long long ib = (long long)n.y * pitch + n.x;
    const int xl = n.dx > 0 ? n.x : n.x - 1;
    if (n.dy == 0 && n.dx != 0 && (xl & 1) == 0) {
        using V2 = typename std::conditional<sizeof(R) == 4, float2, double2>::type;
        const R* row = buf + (long long)n.y * pitch + xl;
#pragma unroll
        for (int q = 0; q < 18; ++q) {
            const V2 pr = __ldg(reinterpret_cast<const V2*>(row + q * plane));
            v[q] = n.dx > 0 ? pr.x : pr.y;
            u[q] = n.dx > 0 ? pr.y : pr.x;
        }
    } else {
        load18<R>(buf, plane, ib, v);
        load18<R>(buf, plane, (long long)(n.y + n.dy) * pitch + (n.x + n.dx), u);
    }
    // density (and Neumann total energy) from the bounced-back populations
    R rd, jx, jy, sg;
    lbm::node_sums(v, v + 9, rd, jx, jy, sg);
    const R ux = R(n.ux), uy = R(n.uy);
    Mac<R> mb;
    R rhoE_d;
    if (n.thermal == 0) {
        const R Td = R(n.T) - P.T0;
        const R Ed = P.Cv * Td + R(0.5) * (ux * ux + uy * uy);
        rhoE_d = rd * P.E0 + (P.rho0 + rd) * Ed;
    } else {
        const R rho = P.rho0 + rd;
        const R Fx = P.force_mode ? rho * P.Fx : P.Fx;
        const R Fy = P.force_mode ? rho * P.Fy : P.Fy;
        rhoE_d = sg + R(0.5) * (ux * Fx + uy * Fy);
    }
    lbm::wall_macros(P, rd, ux, uy, rhoE_d, mb);

    // redefined non-equilibrium moments at x_f (and x_ff), extrapolated
    R mt[9], nt[9];
    {
        Mac<R> m;
        node_macros(P, u, m);
        lbm::tilde_neq(P, m, u, u + 9, mt, nt);
        if (n.order == 2) {
            R mt2[9], nt2[9];
            load18<R>(buf, plane, (long long)(n.y + 2 * n.dy) * pitch + (n.x + 2 * n.dx), u);
            node_macros(P, u, m);
            lbm::tilde_neq(P, m, u, u + 9, mt2, nt2);
#pragma unroll
            for (int q = 0; q < 9; ++q) {
                mt[q] = R(2) * mt[q] - mt2[q];
                nt[q] = R(2) * nt[q] - nt2[q];
            }
        }
    }
    lbm::rebuild(P, mb, mt, nt, v, v + 9);
    store18<R>(buf, plane, ib, v);
}

// ------------------------------------------------------------------------
// initialisation, state transfer, macros, reductions
// ------------------------------------------------------------------------

template <typename R>
__global__ void k_init_rest(const InstDesc* D, int b) {
    const Params<R>& P = dparams<R>(D);
    const long long nn = (long long)D->nx * D->ny;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nn;
         t += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(t / D->nx), x = (int)(t % D->nx);
        Mac<R> m;
        lbm::wall_macros(P, R(0), R(0), R(0), R(0), m);
        R v[18];
        lbm::equilibrium(P, m, v, v + 9);
        store18<R>(reinterpret_cast<R*>(D->buf[b]), D->plane, (long long)y * D->pitch + x, v);
    }
}

template <typename R>
__global__ void k_init_macros(const InstDesc* D, int b, const double* __restrict__ rho,
                              const double* __restrict__ ux, const double* __restrict__ uy,
                              const double* __restrict__ T) {
    const Params<double>& Pd = D->pd;
    const Params<R>& P = dparams<R>(D);
    const long long nn = (long long)D->nx * D->ny;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nn;
         t += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(t / D->nx), x = (int)(t % D->nx);
        const double rd = rho[t] - Pd.rho0;
        const double u = ux[t], vv = uy[t];
        const double Ed = Pd.Cv * (T[t] - Pd.T0) + 0.5 * (u * u + vv * vv);
        const double rhoE_d = rd * Pd.E0 + rho[t] * Ed;
        Mac<R> m;
        lbm::wall_macros(P, R(rd), R(u), R(vv), R(rhoE_d), m);
        R v[18];
        lbm::equilibrium(P, m, v, v + 9);
        store18<R>(reinterpret_cast<R*>(D->buf[b]), D->plane, (long long)y * D->pitch + x, v);
    }
}

// plane q of buffer b <-> dense FP64 array [ny][nx] of full values (deviation + rest)
template <typename R>
__global__ void k_get_plane(const InstDesc* D, int b, int q, double rest, double* __restrict__ out) {
    const long long nn = (long long)D->nx * D->ny;
    const R* base = reinterpret_cast<const R*>(D->buf[b]) + q * D->plane;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nn;
         t += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(t / D->nx), x = (int)(t % D->nx);
        out[t] = (double)base[(long long)y * D->pitch + x] + rest;
    }
}

template <typename R>
__global__ void k_set_plane(const InstDesc* D, int b, int q, double rest, const double* __restrict__ in) {
    const long long nn = (long long)D->nx * D->ny;
    R* base = reinterpret_cast<R*>(D->buf[b]) + q * D->plane;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nn;
         t += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(t / D->nx), x = (int)(t % D->nx);
        base[(long long)y * D->pitch + x] = (R)(in[t] - rest);
    }
}

// Plane-by-plane copy of a DF buffer into another context's buffer of the
// same extents, converting the storage type (both hold deviations from the
// same rest equilibrium).
template <typename Rs, typename Rd>
__global__ void k_copy_state(const Rs* __restrict__ src, long long splane, int spitch, Rd* __restrict__ dst,
                             long long dplane, int dpitch, int nx, int ny) {
    const long long nn = (long long)nx * ny, total = 18 * nn;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        const long long q = i / nn, r = i - q * nn;
        const int y = (int)(r / nx), x = (int)(r - (long long)y * nx);
        dst[q * dplane + (long long)y * dpitch + x] = (Rd)src[q * splane + (long long)y * spitch + x];
    }
}

// FP64 macros of one node of an R-typed buffer.
template <typename R>
__device__ __forceinline__ void macros_fp64(const InstDesc* D, const R* buf, int x, int y, Mac<double>& m) {
    R v[18];
    load18(buf, D->plane, (long long)y * D->pitch + x, v);
    double w[18];
#pragma unroll
    for (int q = 0; q < 18; ++q) w[q] = (double)v[q];
    double rd, jx, jy, sg;
    lbm::node_sums(w, w + 9, rd, jx, jy, sg);
    lbm::macros(D->pd, rd, jx, jy, sg, m);
}

template <typename R>
__global__ void k_macros(const InstDesc* D, int b, double* rho, double* ux, double* uy, double* T,
                         double* p) {
    const long long nn = (long long)D->nx * D->ny;
    const R* buf = reinterpret_cast<const R*>(D->buf[b]);
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nn;
         t += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(t / D->nx), x = (int)(t % D->nx);
        Mac<double> m;
        macros_fp64(D, buf, x, y, m);
        if (rho) rho[t] = m.rho;
        if (ux) ux[t] = m.ux;
        if (uy) uy[t] = m.uy;
        if (T) T[t] = m.T;
        if (p) p[t] = D->pd.p0 + m.p_d;
    }
}

constexpr int kDiagSlots = 10;
constexpr int kDiagBlocks = 304;   // 2 per SM on a 152-SM part; fixed for a deterministic order
constexpr int kDiagThreads = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}

// Per-block FP64 partial sums (slot 8 is a maximum) into partials[block][kDiagSlots]:
// block blk of nblk, grid-stride over the lattice's nodes.  k_diag and the
// batched k_diag_batch run this with the same decomposition, so a lattice's
// diagnostics are the same bits alone or batched.
template <typename R>
__device__ __forceinline__ void diag_partials(const InstDesc* D, int b, double* __restrict__ snap, int take_snapshot,
                                              int have_snapshot, double* __restrict__ partials, int blk, int nblk) {
    const long long nn = (long long)D->nx * D->ny;
    const R* buf = reinterpret_cast<const R*>(D->buf[b]);
    double acc[kDiagSlots];
#pragma unroll
    for (int s = 0; s < kDiagSlots; ++s) acc[s] = 0.0;
    const double Lx = D->px ? (double)D->nx : (double)(D->nx - 1);
    const double Ly = D->py ? (double)D->ny : (double)(D->ny - 1);
    for (long long t = blk * (long long)blockDim.x + threadIdx.x; t < nn; t += (long long)nblk * blockDim.x) {
        const int y = (int)(t / D->nx), x = (int)(t % D->nx);
        Mac<double> m;
        macros_fp64(D, buf, x, y, m);
        const bool bad = !(isfinite(m.rho) && isfinite(m.T) && isfinite(m.ux) && isfinite(m.uy));
        if (bad) { acc[7] += 1.0; continue; }
        const double wx = (!D->px && (x == 0 || x == D->nx - 1)) ? 0.5 : 1.0;
        const double wy = (!D->py && (y == 0 || y == D->ny - 1)) ? 0.5 : 1.0;
        const double p = D->pd.p0 + m.p_d;
        acc[0] += m.rho_d;
        acc[1] += m.rhoE_d;
        acc[2] += wx * wy * p / (D->pd.p0 * Lx * Ly);
        const double u2 = m.ux * m.ux + m.uy * m.uy;
        if (have_snapshot) {
            const double dux = m.ux - snap[t], duy = m.uy - snap[nn + t], dT = m.T - snap[2 * nn + t];
            acc[3] += dux * dux + duy * duy;
            acc[5] += dT * dT;
        }
        acc[4] += u2;
        acc[6] += m.T_d * m.T_d;
        acc[8] = fmax(acc[8], sqrt(u2));
        acc[9] += m.T;
        if (take_snapshot) {
            snap[t] = m.ux;
            snap[nn + t] = m.uy;
            snap[2 * nn + t] = m.T;
        }
    }
    __shared__ double red[kDiagThreads / 32][kDiagSlots];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int s = 0; s < kDiagSlots; ++s) {
        const double v = (s == 8) ? warp_max(acc[s]) : warp_sum(acc[s]);
        if (lane == 0) red[wid][s] = v;
    }
    __syncthreads();
    if (threadIdx.x < kDiagSlots) {
        const int s = threadIdx.x;
        double v = red[0][s];
        for (int k = 1; k < kDiagThreads / 32; ++k) v = (s == 8) ? fmax(v, red[k][s]) : v + red[k][s];
        partials[blk * kDiagSlots + s] = v;
    }
}

template <typename R>
__global__ void __launch_bounds__(kDiagThreads) k_diag(const InstDesc* D, int b, double* __restrict__ snap,
                                                       int take_snapshot, int have_snapshot,
                                                       double* __restrict__ partials) {
    diag_partials<R>(D, b, snap, take_snapshot, have_snapshot, partials, blockIdx.x, gridDim.x);
}

// One lattice of a batched diagnostics pass (lbm_batch_diagnostics).
struct DiagJob {
    const InstDesc* D;
    double* snap;
    double* partials;
    const unsigned int* status;
    int b, have;
};

// Every lattice of one storage precision at once: blockIdx.y picks the job.
template <typename R>
__global__ void __launch_bounds__(kDiagThreads) k_diag_batch(const DiagJob* __restrict__ jobs, int take_snapshot) {
    const DiagJob j = jobs[blockIdx.y];
    diag_partials<R>(j.D, j.b, j.snap, take_snapshot, j.have, j.partials, blockIdx.x, gridDim.x);
}

__global__ void k_diag_final(const double* __restrict__ partials, int nblocks, double* __restrict__ out) {
    const int s = threadIdx.x;
    if (s >= kDiagSlots) return;
    double v = 0.0;
    for (int k = 0; k < nblocks; ++k) v = (s == 8) ? fmax(v, partials[k * kDiagSlots + s]) : v + partials[k * kDiagSlots + s];
    out[s] = v;
}

// Block b finishes job b: its kDiagSlots sums, then its status word, into
// out[b][kDiagSlots + 1], in the order k_diag_final uses.
__global__ void k_diag_final_batch(const DiagJob* __restrict__ jobs, int nblocks, double* __restrict__ out) {
    const DiagJob j = jobs[blockIdx.x];
    const int s = threadIdx.x;
    double* o = out + (size_t)blockIdx.x * (kDiagSlots + 1);
    if (s == kDiagSlots) o[s] = (double)*j.status;
    if (s >= kDiagSlots) return;
    double v = 0.0;
    for (int k = 0; k < nblocks; ++k) v = (s == 8) ? fmax(v, j.partials[k * kDiagSlots + s]) : v + j.partials[k * kDiagSlots + s];
    o[s] = v;
}

// ------------------------------------------------------------------------
// arithmetic-rate probes (lbm_peak_rates)
// ------------------------------------------------------------------------

// Dependent multiply-add chains, kProbeChains independent ones per thread,
// kProbeIters steps each; the result is written so that nothing is elided.
constexpr int kProbeIters = 2048;
constexpr int kProbeChains = 4;

__global__ void k_probe_fp64(double* out) {
    double a[kProbeChains];
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) a[c] = 1.0 + 1e-3 * (threadIdx.x + c);
    const double b = 0.9999999, d = 1e-7;
    for (int i = 0; i < kProbeIters; ++i)
#pragma unroll
        for (int c = 0; c < kProbeChains; ++c) a[c] = fma(a[c], b, d);
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) s += a[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_probe_fp32(float* out) {
    float a[kProbeChains];
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) a[c] = 1.0f + 1e-3f * (threadIdx.x + c);
    const float b = 0.9999999f, d = 1e-7f;
    for (int i = 0; i < kProbeIters; ++i)
#pragma unroll
        for (int c = 0; c < kProbeChains; ++c) a[c] = fmaf(a[c], b, d);
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) s += a[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_probe_ff64(float* out) {
    ff64 a[kProbeChains];
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) a[c] = ff64(1.0f + 1e-3f * (threadIdx.x + c), 0.0f);
    const ff64 b(0.9999999f, 1e-12f), d(1e-7f, 0.0f);
    for (int i = 0; i < kProbeIters; ++i)
#pragma unroll
        for (int c = 0; c < kProbeChains; ++c) a[c] = a[c] * b + d;
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) s += a[c].hi + a[c].lo;
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// ------------------------------------------------------------------------
// conserved sums with statically allocated scratch (lbm_conserved_sums_static)
// ------------------------------------------------------------------------

// Block partials of lbm_conserved_sums_static live in this file-scope array
// instead of caller- or library-allocated memory.  Every GPU that loads the
// library holds it until the process exits.  Each block covers a fixed,
// contiguous range of kStaticNodesPerBlock nodes, so the lattice size sets
// how many slots are used.
constexpr int kStaticBlocks = 2048;
constexpr int kStaticThreads = 256;
constexpr long long kStaticNodesPerBlock = 32768;
static __device__ __align__(256) double g_static_partials[kStaticBlocks * 4];

template <typename R>
__global__ void __launch_bounds__(kStaticThreads) k_sums_static(const InstDesc* D, int b, double* __restrict__ partials) {
    const long long nn = (long long)D->nx * D->ny;
    const R* buf = reinterpret_cast<const R*>(D->buf[b]);
    const long long lo = blockIdx.x * kStaticNodesPerBlock;
    const long long hi = lo + kStaticNodesPerBlock < nn ? lo + kStaticNodesPerBlock : nn;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (long long t = lo + threadIdx.x; t < hi; t += kStaticThreads) {
        const int y = (int)(t / D->nx), x = (int)(t % D->nx);
        R v[18];
        load18(buf, D->plane, (long long)y * D->pitch + x, v);
        double w[18];
#pragma unroll
        for (int q = 0; q < 18; ++q) w[q] = (double)v[q];
        double rd, jx, jy, sg;
        lbm::node_sums(w, w + 9, rd, jx, jy, sg);
        acc[0] += rd;
        acc[1] += jx;
        acc[2] += jy;
        acc[3] += sg;
    }
    __shared__ double red[kStaticThreads / 32][4];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        const double v = warp_sum(acc[s]);
        if (lane == 0) red[wid][s] = v;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        double v = 0.0;
        for (int k = 0; k < kStaticThreads / 32; ++k) v += red[k][threadIdx.x];
        partials[blockIdx.x * 4 + threadIdx.x] = v;
    }
}

__global__ void k_sums_static_final(const InstDesc* D, const double* __restrict__ partials, int nblocks,
                                    double* __restrict__ out4) {
    const int s = threadIdx.x;
    if (s >= 4) return;
    double v = 0.0;
    for (int k = 0; k < nblocks; ++k) v += partials[k * 4 + s];
    const double nn = (double)D->nx * D->ny;
    // the rest equilibria carry rho0 and rho0 E0 per node and no momentum
    if (s == 0) v += nn * D->pd.rho0;
    if (s == 3) v += nn * D->pd.rho0 * D->pd.E0;
    out4[s] = v;
}

// Mean Nusselt number through one wall: one block, fixed-order tree.
template <typename R>
__global__ void __launch_bounds__(1024) k_nusselt(const InstDesc* D, int b, int wall, double dT, double* out) {
    const R* buf = reinterpret_cast<const R*>(D->buf[b]);
    const int nx = D->nx, ny = D->ny;
    const int len = (wall >= 2) ? ny : nx;
    const Params<double>& P = D->pd;
    double acc = 0.0;
    for (int t = threadIdx.x; t < len; t += blockDim.x) {
        int x0, y0, dx, dy;
        if (wall == 0) { x0 = t; y0 = 0; dx = 0; dy = 1; }
        else if (wall == 1) { x0 = t; y0 = ny - 1; dx = 0; dy = -1; }
        else if (wall == 2) { x0 = 0; y0 = t; dx = 1; dy = 0; }
        else { x0 = nx - 1; y0 = t; dx = -1; dy = 0; }
        Mac<double> m0, m1, m2;
        macros_fp64(D, buf, x0, y0, m0);
        macros_fp64(D, buf, x0 + dx, y0 + dy, m1);
        macros_fp64(D, buf, x0 + 2 * dx, y0 + 2 * dy, m2);
        const double dTdn = (-3.0 * m0.T + 4.0 * m1.T - m2.T) * 0.5;
        const double lam = P.lam_fac * lbm::viscosity(P, m0.T);
        const double wgt = (t == 0 || t == len - 1) ? 0.5 : 1.0;
        acc += wgt * (-lam * dTdn);
    }
    __shared__ double red[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    acc = warp_sum(acc);
    if (lane == 0) red[wid] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double v = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) v += red[k];
        const double lam0 = P.lam_fac * P.mu0;
        out[0] = v / (lam0 * dT);
    }
}

// ------------------------------------------------------------------------
// host side
// ------------------------------------------------------------------------

thread_local std::string g_err;

lbm_status fail(lbm_status st, const std::string& msg) {
    g_err = msg;
    return st;
}

#define CUDA_TRY(call)                                                                       \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return fail(LBM_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));      \
    } while (0)

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

struct Layout {
    size_t off_desc, off_descs, off_status, off_diag, off_partials, off_bufA, off_bufB, off_snap, off_stage;
    size_t total, buf_bytes;
    int pitch;
    long long plane;
};

Layout layout_for(const lbm_config& c) {
    Layout L{};
    const size_t es = c.precision == LBM_FP32_DEV ? 4 : 8;
    L.pitch = (int)align_up((size_t)c.nx, 32);
    L.plane = (long long)L.pitch * c.ny;
    const size_t nn = (size_t)c.nx * c.ny;
    size_t o = 0;
    L.off_desc = o; o = align_up(o + sizeof(InstDesc), 256);
    L.off_descs = o; o = align_up(o + sizeof(void*), 256);
    L.off_status = o; o = align_up(o + 256, 256);
    L.off_diag = o; o = align_up(o + 16 * sizeof(double), 256);
    L.off_partials = o; o = align_up(o + (size_t)kDiagBlocks * kDiagSlots * sizeof(double), 256);
    L.buf_bytes = align_up((size_t)18 * L.plane * es, 256);
    L.off_bufA = o; o += L.buf_bytes;
    L.off_bufB = o; o += L.buf_bytes;
    L.off_snap = o; o = align_up(o + 3 * nn * sizeof(double), 256);
    L.off_stage = o; o = align_up(o + 5 * nn * sizeof(double), 256);
    L.total = o;
    return L;
}

lbm_status validate(const lbm_config* c) {
    if (!c) return fail(LBM_EINVAL, "null config");
    const int px = c->wall[LBM_WALL_W].periodic != 0, pxe = c->wall[LBM_WALL_E].periodic != 0;
    const int py = c->wall[LBM_WALL_S].periodic != 0, pyn = c->wall[LBM_WALL_N].periodic != 0;
    if (px != pxe || py != pyn) return fail(LBM_EINVAL, "a periodic side must face a periodic side");
    if (c->nx < 1 || c->ny < 1) return fail(LBM_EINVAL, "nx, ny must be >= 1");
    if ((!px && c->nx < 4) || (!py && c->ny < 4)) return fail(LBM_EINVAL, "walled extents need >= 4 nodes");
    if (18LL * (long long)(((c->nx + 31) / 32) * 32) * c->ny >= (1LL << 31))
        return fail(LBM_EINVAL, "lattice too large: 18 planes must fit 32-bit offsets");
    if (c->precision != LBM_FP64 && c->precision != LBM_FP32_DEV) return fail(LBM_EINVAL, "bad precision");
    for (int s = 0; s < 4; ++s) {
        if (c->wall[s].periodic) continue;
        if (c->wall[s].extrap_order != 1 && c->wall[s].extrap_order != 2)
            return fail(LBM_EINVAL, "extrap_order must be 1 or 2");
        if (c->wall[s].thermal != 0 && c->wall[s].thermal != 1) return fail(LBM_EINVAL, "thermal must be 0 or 1");
    }
    if (!(c->tau0 > 0.5) || !(c->rho0 > 0) || !(c->T0 > 0) || !(c->gamma > 1.0) || !(c->Pr > 0))
        return fail(LBM_EINVAL, "need tau0 > 1/2, rho0, T0, Pr > 0, gamma > 1");
    if (!(c->varpi > 0 && c->varpi < 1.0 / 3.0)) return fail(LBM_EINVAL, "varpi must lie in (0, 1/3)");
    if (!(c->bulk_ratio > 0)) return fail(LBM_EINVAL, "bulk_ratio must be > 0");
    if (c->visc_law < 0 || c->visc_law > 2) return fail(LBM_EINVAL, "bad visc_law");
    return LBM_OK;
}

template <typename A, typename B>
void convert_params(const Params<A>& a, Params<B>& b) {
#define CP(f) b.f = (B)a.f
    CP(rho0); CP(T0); CP(E0); CP(Cv); CP(inv_Cv); CP(Rg); CP(eos_a); CP(eos_b); CP(p0); CP(rho0E0_p0);
    CP(rho0Cp0); CP(mu0); CP(inv_T0); CP(visc_S); CP(lam_fac); CP(tj_fac); CP(e_fac); CP(alpha1);
    CP(beta1); CP(alpha2); CP(beta2); CP(kk); CP(hh); CP(bb); CP(gamma1); CP(gamma2); CP(cR11);
    CP(cR17); CP(cR18); CP(cR71); CP(cR77); CP(cR81); CP(cR88); CP(Fx); CP(Fy); CP(cs_b0); CP(dither);
#undef CP
    b.eos = a.eos;
    b.visc = a.visc;
    b.force_mode = a.force_mode;
    b.corrections = a.corrections;
}

// f = M^-1 m (host, FP64) for the rest equilibria.
void host_inverse_moments(const double* m, double* f) { lbm::inverse_moments<double>(m, f); }

}  // namespace

struct lbm_ctx {
    lbm_config cfg;
    cudaStream_t stream = nullptr;
    bool own_ws = false;
    char* ws = nullptr;
    size_t ws_bytes = 0;
    Layout L{};
    InstDesc h{};
    InstDesc* d_desc = nullptr;
    InstDesc** d_descs = nullptr;
    unsigned int* d_status = nullptr;
    long long* d_counter = nullptr;  // absolute step read by the fused kernel
    double* d_diag = nullptr;
    double* d_partials = nullptr;
    double* d_snap = nullptr;
    double* d_stage = nullptr;
    Work* d_work = nullptr;
    int n_work = 0, bx = 128, by = 0, pair = 0;
    bool tile_set = false;  // launch shape chosen by lbm_set_tile, kept in batches
    int mc = 0;             // model class of the fused kernel (lbm::MODEL_*), set with the EOS
    int round_mode = LBM_ROUND_STOCHASTIC;  // rounding of FP32 stores (lbm_set_rounding)
    int device = 0;         // device current at lbm_create, which holds the workspace
    BWork* d_bwork = nullptr;
    int n_bwork = 0;
    long steps = 0;
    bool eos_set = false, have_snap = false;
    lbm_status sticky = LBM_OK;
    double derived[8] = {0};
    double f_rest[9] = {0}, g_rest[9] = {0};
    std::vector<Work> h_work;
    std::vector<BWork> h_bwork;
};

// Fused-kernel variants: strips of 32, 64, 128 columns, one node per thread
// (indices 0-2, pair = 0); strips of 64, 128, 256 columns, two nodes per
// thread in packed FP32 keeping the row macros in registers (indices 3-5,
// pair = 1) or recomputing them at collision time (indices 6-8, pair = 2);
// one node per thread recomputing the macros, fewer registers (indices 9-11,
// pair = 3); one autonomous warp per 30 columns, 1, 2 or 4 warps per CTA
// (indices 12-14, pair = 4); one autonomous warp per 60 columns, two nodes
// per lane in packed FP32 (indices 15-17, pair = 5).  Variants 3-11 and
// 15-17 need FP32 storage.
constexpr int kVariants = 18;
constexpr int kModels = 2;  // model classes: lbm::MODEL_ANY, lbm::MODEL_CAVITY
// Lattices below this many nodes keep the generic instance even with the
// cavity model: they are latency-bound, and batches of them (the serving
// mix) then stay one launch per shape.
constexpr long long kModelMinNodes = 32768;

// The launches of one time step over a set of members: launch groups
// [precision][variant][model class] as ranges of the batch's work table,
// wall-pass ranges [precision] of its wall table, and the step counter
// that the set's last wall-pass launch advances and its fused launches read.
struct LaunchSet {
    int w_off[2][kVariants][kModels] = {}, w_cnt[2][kVariants][kModels] = {};
    int b_off[2] = {0, 0}, b_cnt[2] = {0, 0};
    long long* counter = nullptr;
};

struct lbm_batch {
    std::vector<lbm_ctx*> ctxs;
    std::vector<int> models;  // each member's model class when the launch groups were built
    cudaStream_t stream = nullptr;
    InstDesc** d_descs = nullptr;
    Work* d_work = nullptr;
    BWork* d_bwork = nullptr;
    LaunchSet set;                   // every member's launches of one time step
    long steps = 0;
    int graph_steps = 0;
    cudaGraphExec_t graph = nullptr;
    long long* d_counter = nullptr;  // the batch's step counter, advanced on the device
    DiagJob* d_jobs = nullptr;       // lbm_batch_diagnostics: one job per member, FP32 members first
    double* d_diag_out = nullptr;    // [member][kDiagSlots + 1] sums and status word
    std::vector<int> diag_order;     // members in job order
    unsigned int* d_status_all = nullptr;  // lbm_batch_macros: every member's status word
};

namespace {

// Work items of one lattice: strips of bx columns, each cut into
// ceil(ny / by) runs of rows whose lengths differ by at most one.
std::vector<Work> make_work(const lbm_config& c, int inst, int bx, int by, int par, long long step0) {
    std::vector<Work> v;
    const long long nruns = (c.ny + by - 1) / by;
    for (long long r = 0; r < nruns; ++r)
        for (int x0 = 0; x0 < c.nx; x0 += bx) {
            Work w{};
            w.inst = inst;
            w.x0 = x0;
            w.y0 = (int)(r * c.ny / nruns);
            w.y1 = (int)((r + 1) * c.ny / nruns);
            w.par = par;
            w.dir = (int)(r & 1);
            w.step0 = step0;
            v.push_back(w);
        }
    return v;
}

// Shorter runs at the end of a launch: the CTAs of one launch start as
// resident slots free up, so the launch ends when the last ones finish, and
// with runs of equal length the GPU idles for up to one run at the end.
// The last `resident` work items (one fill of the GPU) are cut into up to
// four runs of at least 6 rows each (shorter runs re-stage too many halo
// rows), placed last; that shortens the idle end to about a quarter of a
// run.  Measured on the 96-cavity batch (runs of 32 rows): fused launch
// 1.138 -> 1.123 ms; 16 cavities of 1024^2: 0.503 -> 0.488 ms.  Which CTA
// updates a node does not change its arithmetic, so the results are the
// same bits.
void split_tail(std::vector<Work>& v, long long resident) {
    if (resident <= 0 || (long long)v.size() <= resident) return;
    const size_t first = v.size() - (size_t)resident;
    std::vector<Work> tail(v.begin() + first, v.end());
    v.resize(first);
    for (int part = 0; part < 4; ++part)
        for (const Work& w : tail) {
            const int rows = w.y1 - w.y0;
            const int parts = std::max(1, std::min(4, rows / 6));
            if (part >= parts) continue;
            Work u = w;
            u.y0 = w.y0 + rows * part / parts;
            u.y1 = w.y0 + rows * (part + 1) / parts;
            u.dir = (w.dir + part) & 1;
            v.push_back(u);
        }
}

std::vector<BWork> make_bwork(const lbm_config& c, int inst, int par) {
    std::vector<BWork> v;
    const int px = c.wall[LBM_WALL_W].periodic != 0, py = c.wall[LBM_WALL_S].periodic != 0;
    const int n = wall_count(c.nx, c.ny, px, py);
    for (int k0 = 0; k0 < n; k0 += 128) {
        BWork b{};
        b.inst = inst;
        b.k0 = k0;
        b.cnt = std::min(128, n - k0);
        b.par = par;
        v.push_back(b);
    }
    return v;
}

// A fully periodic lattice has no wall nodes; one empty item keeps a wall-pass
// launch in every step so that it can advance the step counter.
void ensure_tick(std::vector<BWork>& v, int inst, int par) {
    if (v.empty()) {
        BWork b{};
        b.inst = inst;
        b.par = par;
        v.push_back(b);
    }
}

// Default launch shape.  Lattices up to 160 columns wide take warp strips
// of 30 columns (pair 4, same bits as pair 0): they waste fewer lanes there
// and give small lattices more CTAs.  Wider FP32 lattices of the heated-
// cavity model class take paired block strips of 128 columns (pair 1): two
// nodes per thread in packed FP32 halve the arithmetic's issue slots (4096^2:
// 0.49 ms against 0.55 ms for block strips; 96-cavity batch: 1.30 ms against
// 1.39 ms per step).  All others take block strips of 128 columns (pair 0),
// which also suit FP64, bound by the FP64 pipe.  The model class is known
// once the EOS is set, so lbm_set_eos applies the shape.
void default_shape(const lbm_config& c, int mc, int& bx, int& pair) {
    if (c.nx <= 160) { bx = 30; pair = 4; }
    else if (c.precision == LBM_FP32_DEV && mc == lbm::MODEL_CAVITY) { bx = 128; pair = 1; }
    else { bx = 128; pair = 0; }
}

// Longest run of rows per CTA: the best measured on a 4096^2 (FP32) or
// 2048^2 (FP64) lattice and on the 96-cavity batch (longer runs lose DRAM
// and L2 locality between CTAs resident at the same time, shorter ones
// re-stage more halo rows).  Paired block strips: 32 rows on the 96-cavity
// batch (1.285 ms per step against 1.302 ms with 24).
int batch_rows(const lbm_config& c, int pair) {
    const bool f32 = c.precision == LBM_FP32_DEV;
    const int by = pair == 0 ? (f32 ? 24 : 8) : pair == 1 ? 32 : (pair == 5 ? 16 : 24);
    return std::min(c.ny, by);
}

long long cta_count(const lbm_config& c, int bx, int by) {
    return (long long)((c.nx + bx - 1) / bx) * ((c.ny + by - 1) / by);
}

// Rows per run for a lattice launched on its own.  Block and warp strips:
// ny / 128, between 1 and the longest run (measured optimum on square FP32
// lattices: 1-2 rows at 256^2, 4 at 512^2, 8 at 1024^2, 12-16 at 2048^2, 24
// at 4096^2).  Paired block strips: 3 ny / 512, between 1 and 12 (measured:
// 2-4 at 512^2, 6 at 1024^2, 8-12 at 2048^2, 12 at 4096^2).  A small
// lattice is latency-bound and gains more from spreading over more SMs than
// it loses re-staging halo rows.
int default_rows(const lbm_config& c, int pair) {
    if (pair == 1) return std::max(1, std::min(std::min(batch_rows(c, pair), 12), c.ny * 3 / 512));
    return std::max(1, std::min(batch_rows(c, pair), c.ny / 128));
}

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime.
EncodeTiledFn encode_tiled() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    return fn;
}

// Tensor maps of the row windows of the warp-strip kernels over both DF
// buffers, viewed as the tensor [18 planes][ny rows][pitch columns].
lbm_status encode_windows(lbm_ctx* c) {
    EncodeTiledFn enc = encode_tiled();
    if (!enc) return fail(LBM_ECUDA, "cuTensorMapEncodeTiled is not available from the driver");
    const bool f32 = c->cfg.precision == LBM_FP32_DEV;
    const cuuint64_t es = f32 ? 4 : 8;
    const cuuint64_t dims[3] = {(cuuint64_t)c->L.pitch, (cuuint64_t)c->cfg.ny, 18};
    const cuuint64_t strides[2] = {(cuuint64_t)c->L.pitch * es, (cuuint64_t)c->L.plane * es};
    const cuuint32_t estr[3] = {1, 1, 1};
    const int E = (int)(16 / es);
    memset(c->h.tmap, 0, sizeof(c->h.tmap));
    for (int k = 0; k < kTmaps; ++k) {
        if (k == 1 && !f32) continue;  // paired warp strips are FP32 only
        const int width = k < 2 ? kWinCols[k] : (32 << (k - 2)) + 2 * E;
        const cuuint32_t box[3] = {(cuuint32_t)width, 1, 18};
        for (int b = 0; b < 2; ++b) {
            const CUresult r = enc(&c->h.tmap[k][b], f32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64,
                                   3, c->h.buf[b], dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                   CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (r != CUDA_SUCCESS)
                return fail(LBM_ECUDA, "cuTensorMapEncodeTiled failed (code " + std::to_string((int)r) + ")");
        }
    }
    return LBM_OK;
}

long long resident_ctas(int vi, bool fp32);
int variant_index(int bx, int pair);
bool is_fp32(const lbm_ctx* c);

lbm_status upload_work(lbm_ctx* c) {
    if (c->d_work) { cudaFree(c->d_work); c->d_work = nullptr; }
    c->h_work = make_work(c->cfg, 0, c->bx, c->by, 0, 0);
    split_tail(c->h_work, resident_ctas(variant_index(c->bx, c->pair), is_fp32(c)));
    c->n_work = (int)c->h_work.size();
    CUDA_TRY(cudaMalloc(&c->d_work, c->h_work.size() * sizeof(Work)));
    CUDA_TRY(cudaMemcpyAsync(c->d_work, c->h_work.data(), c->h_work.size() * sizeof(Work),
                             cudaMemcpyHostToDevice, c->stream));
    return LBM_OK;
}

template <typename R, int BX, bool KEEP = true, int MC = lbm::MODEL_ANY>
cudaError_t configure_collide() {
    constexpr int S = FusedTraits<R, BX>::S;
    cudaError_t e = cudaFuncSetAttribute(k_collide_stream<R, BX, S, KEEP, MC>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FusedSmem<R, BX, S>::bytes);
    if (e != cudaSuccess) return e;
    // prefer shared memory over L1: the row stages, not L1, feed the kernel
    return cudaFuncSetAttribute(k_collide_stream<R, BX, S, KEEP, MC>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                (int)cudaSharedmemCarveoutMaxShared);
}

template <typename R, int NW, int MC = lbm::MODEL_ANY>
cudaError_t configure_warp() {
    constexpr int S = WarpTraits<R>::S;
    cudaError_t e = cudaFuncSetAttribute(k_collide_warp<R, NW, S, MC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)WarpSmem<R, NW, S>::bytes);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_collide_warp<R, NW, S, MC>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                (int)cudaSharedmemCarveoutMaxShared);
}

template <typename R, int MC>
cudaError_t configure_model() {
    cudaError_t e = configure_collide<R, 32, true, MC>();
    if (e == cudaSuccess) e = configure_collide<R, 64, true, MC>();
    if (e == cudaSuccess) e = configure_collide<R, 128, true, MC>();
    if (e == cudaSuccess) e = configure_warp<R, 1, MC>();
    if (e == cudaSuccess) e = configure_warp<R, 2, MC>();
    if (e == cudaSuccess) e = configure_warp<R, 4, MC>();
    return e;
}
template <typename R>
cudaError_t configure_models() {
    return configure_model<R, lbm::MODEL_CAVITY>();
}

template <int NW>
cudaError_t configure_warp2() {
    cudaError_t e = cudaFuncSetAttribute(k_collide_warp2<NW, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)Warp2Smem<NW, 3>::bytes);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_collide_warp2<NW, 3>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                (int)cudaSharedmemCarveoutMaxShared);
}

template <int BX, bool KEEP, int MC = lbm::MODEL_ANY>
cudaError_t configure_pair() {
    cudaError_t e = cudaFuncSetAttribute(k_collide_pair<BX, KEEP, MC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)PairSmem<BX>::bytes);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_collide_pair<BX, KEEP, MC>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                (int)cudaSharedmemCarveoutMaxShared);
}

// Dynamic shared memory above 48 KB must be enabled per kernel before its
// first launch (and before any graph capture that contains it).
lbm_status configure_kernels() {
    static int done = 0;
    if (done) return LBM_OK;
    cudaError_t e = configure_collide<float, 32>();
    if (e == cudaSuccess) e = configure_collide<float, 64>();
    if (e == cudaSuccess) e = configure_collide<float, 128>();
    if (e == cudaSuccess) e = configure_collide<float, 32, false>();
    if (e == cudaSuccess) e = configure_collide<float, 64, false>();
    if (e == cudaSuccess) e = configure_collide<float, 128, false>();
    if (e == cudaSuccess) e = configure_pair<64, true>();
    if (e == cudaSuccess) e = configure_pair<128, true>();
    if (e == cudaSuccess) e = configure_pair<256, true>();
    if (e == cudaSuccess) e = configure_pair<64, false>();
    if (e == cudaSuccess) e = configure_pair<128, false>();
    if (e == cudaSuccess) e = configure_pair<256, false>();
    if (e == cudaSuccess) e = configure_collide<double, 32>();
    if (e == cudaSuccess) e = configure_collide<double, 64>();
    if (e == cudaSuccess) e = configure_collide<double, 128>();
    if (e == cudaSuccess) e = configure_warp<float, 1>();
    if (e == cudaSuccess) e = configure_warp<float, 2>();
    if (e == cudaSuccess) e = configure_warp<float, 4>();
    if (e == cudaSuccess) e = configure_warp<double, 1>();
    if (e == cudaSuccess) e = configure_warp<double, 2>();
    if (e == cudaSuccess) e = configure_warp<double, 4>();
    // the one-node-per-thread shapes, specialised for the heated-cavity models
    if (e == cudaSuccess) e = configure_models<float>();
    if (e == cudaSuccess) e = configure_models<double>();
    if (e == cudaSuccess) e = configure_pair<64, true, lbm::MODEL_CAVITY>();
    if (e == cudaSuccess) e = configure_pair<128, true, lbm::MODEL_CAVITY>();
    if (e == cudaSuccess) e = configure_pair<256, true, lbm::MODEL_CAVITY>();
    if (e == cudaSuccess) e = configure_warp2<1>();
    if (e == cudaSuccess) e = configure_warp2<2>();
    if (e == cudaSuccess) e = configure_warp2<4>();
    if (e != cudaSuccess) return fail(LBM_ECUDA, std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e));
    done = 1;
    return LBM_OK;
}

template <typename K>
int occupancy_of(K kernel, int threads, size_t smem) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, threads, smem) != cudaSuccess) n = 1;
    return std::max(n, 1);
}
template <typename R, int BX, bool KEEP>
int occ_collide() {
    constexpr int S = FusedTraits<R, BX>::S;
    return occupancy_of(k_collide_stream<R, BX, S, KEEP>, BX, FusedSmem<R, BX, S>::bytes);
}
template <int BX, bool KEEP>
int occ_pair() { return occupancy_of(k_collide_pair<BX, KEEP>, BX / 2, PairSmem<BX>::bytes); }
template <typename R, int NW>
int occ_warp() {
    constexpr int S = WarpTraits<R>::S;
    return occupancy_of(k_collide_warp<R, NW, S>, 32 * NW, WarpSmem<R, NW, S>::bytes);
}
template <int NW>
int occ_warp2() { return occupancy_of(k_collide_warp2<NW, 3>, 32 * NW, Warp2Smem<NW, 3>::bytes); }

int variant_per_sm(int vi, bool fp32) {
    switch (vi) {
    case 0: return fp32 ? occ_collide<float, 32, true>() : occ_collide<double, 32, true>();
    case 1: return fp32 ? occ_collide<float, 64, true>() : occ_collide<double, 64, true>();
    case 3: return occ_pair<64, true>();
    case 4: return occ_pair<128, true>();
    case 5: return occ_pair<256, true>();
    case 6: return occ_pair<64, false>();
    case 7: return occ_pair<128, false>();
    case 8: return occ_pair<256, false>();
    case 9: return occ_collide<float, 32, false>();
    case 10: return occ_collide<float, 64, false>();
    case 11: return occ_collide<float, 128, false>();
    case 12: return fp32 ? occ_warp<float, 1>() : occ_warp<double, 1>();
    case 13: return fp32 ? occ_warp<float, 2>() : occ_warp<double, 2>();
    case 14: return fp32 ? occ_warp<float, 4>() : occ_warp<double, 4>();
    case 15: return occ_warp2<1>();
    case 16: return occ_warp2<2>();
    case 17: return occ_warp2<4>();
    default: return fp32 ? occ_collide<float, 128, true>() : occ_collide<double, 128, true>();
    }
}

// CTAs of a variant that the whole GPU holds at once (cached per variant).
long long resident_ctas(int vi, bool fp32) {
    static std::mutex mu;
    static long long cache[2][kVariants] = {{0}};
    std::lock_guard<std::mutex> g(mu);
    long long& r = cache[fp32 ? 1 : 0][vi];
    if (!r) {
        int dev = 0, sms = 152;
        if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        r = (long long)variant_per_sm(vi, fp32) * std::max(sms, 1);
    }
    return r;
}

template <typename R, int BX, bool KEEP = true, int MC = lbm::MODEL_ANY>
void launch_collide_bx(const Work* work, int n, InstDesc* const* descs, int par, const long long* counter,
                       cudaStream_t s) {
    constexpr int S = FusedTraits<R, BX>::S;
    k_collide_stream<R, BX, S, KEEP, MC><<<n, BX, FusedSmem<R, BX, S>::bytes, s>>>(work, descs, par, counter);
}

template <typename R, int NW, int MC = lbm::MODEL_ANY>
void launch_warp_nw(const Work* work, int n, InstDesc* const* descs, int par, const long long* counter,
                    cudaStream_t s) {
    constexpr int S = WarpTraits<R>::S;
    k_collide_warp<R, NW, S, MC><<<n, 32 * NW, WarpSmem<R, NW, S>::bytes, s>>>(work, descs, par, counter);
}

template <int NW>
void launch_warp2_nw(const Work* work, int n, InstDesc* const* descs, int par, const long long* counter,
                     cudaStream_t s) {
    constexpr int S = 3;
    k_collide_warp2<NW, S><<<n, 32 * NW, Warp2Smem<NW, S>::bytes, s>>>(work, descs, par, counter);
}

template <int BX, bool KEEP, int MC = lbm::MODEL_ANY>
void launch_pair_bx(const Work* work, int n, InstDesc* const* descs, int par, const long long* counter,
                    cudaStream_t s) {
    k_collide_pair<BX, KEEP, MC><<<n, BX / 2, PairSmem<BX>::bytes, s>>>(work, descs, par, counter);
}

static const int kVariantWidth[kVariants] = {32, 64, 128, 64, 128, 256, 64, 128, 256, 32, 64, 128, 30, 60, 120,
                                            60, 120, 240};
static const int kVariantPair[kVariants] = {0, 0, 0, 1, 1, 1, 2, 2, 2, 3, 3, 3, 4, 4, 4, 5, 5, 5};

int variant_index(int bx, int pair) {
    for (int v = 0; v < kVariants; ++v)
        if (kVariantWidth[v] == bx && kVariantPair[v] == pair) return v;
    return -1;
}

// Model class a launch of `variant` can use: the shapes that keep the row
// macros (block strips, variants 0-2; paired block strips, variants 3-5;
// warp strips, variants 12-14) have instances specialised for the
// heated-cavity model (the one-node-per-thread ones still give the same bits
// for a lattice); every other shape runs the generic instance.
int launch_model(int variant, int mc) {
    return (variant <= 5 || (variant >= 12 && variant <= 14)) ? mc : lbm::MODEL_ANY;
}

template <typename R, int MC>
void launch_model_variant(const Work* work, int n, int variant, InstDesc* const* descs, int par,
                          const long long* counter, cudaStream_t s) {
    switch (variant) {
    case 0: launch_collide_bx<R, 32, true, MC>(work, n, descs, par, counter, s); break;
    case 1: launch_collide_bx<R, 64, true, MC>(work, n, descs, par, counter, s); break;
    case 2: launch_collide_bx<R, 128, true, MC>(work, n, descs, par, counter, s); break;
    case 3: launch_pair_bx<64, true, MC>(work, n, descs, par, counter, s); break;
    case 4: launch_pair_bx<128, true, MC>(work, n, descs, par, counter, s); break;
    case 5: launch_pair_bx<256, true, MC>(work, n, descs, par, counter, s); break;
    case 12: launch_warp_nw<R, 1, MC>(work, n, descs, par, counter, s); break;
    case 13: launch_warp_nw<R, 2, MC>(work, n, descs, par, counter, s); break;
    default: launch_warp_nw<R, 4, MC>(work, n, descs, par, counter, s); break;
    }
}

template <typename R>
void launch_collide(const Work* work, int n, int variant, int mc, InstDesc* const* descs, int par,
                    const long long* counter, cudaStream_t s) {
    if (n <= 0) return;
    if (launch_model(variant, mc) == lbm::MODEL_CAVITY) {
        launch_model_variant<R, lbm::MODEL_CAVITY>(work, n, variant, descs, par, counter, s);
        return;
    }
    switch (variant) {
    case 0: launch_collide_bx<R, 32>(work, n, descs, par, counter, s); break;
    case 1: launch_collide_bx<R, 64>(work, n, descs, par, counter, s); break;
    case 3: launch_pair_bx<64, true>(work, n, descs, par, counter, s); break;
    case 4: launch_pair_bx<128, true>(work, n, descs, par, counter, s); break;
    case 5: launch_pair_bx<256, true>(work, n, descs, par, counter, s); break;
    case 6: launch_pair_bx<64, false>(work, n, descs, par, counter, s); break;
    case 7: launch_pair_bx<128, false>(work, n, descs, par, counter, s); break;
    case 8: launch_pair_bx<256, false>(work, n, descs, par, counter, s); break;
    case 9: launch_collide_bx<R, 32, false>(work, n, descs, par, counter, s); break;
    case 10: launch_collide_bx<R, 64, false>(work, n, descs, par, counter, s); break;
    case 11: launch_collide_bx<R, 128, false>(work, n, descs, par, counter, s); break;
    case 12: launch_warp_nw<R, 1>(work, n, descs, par, counter, s); break;
    case 13: launch_warp_nw<R, 2>(work, n, descs, par, counter, s); break;
    case 14: launch_warp_nw<R, 4>(work, n, descs, par, counter, s); break;
    case 15: launch_warp2_nw<1>(work, n, descs, par, counter, s); break;
    case 16: launch_warp2_nw<2>(work, n, descs, par, counter, s); break;
    case 17: launch_warp2_nw<4>(work, n, descs, par, counter, s); break;
    default: launch_collide_bx<R, 128>(work, n, descs, par, counter, s); break;
    }
}

template <typename R>
void launch_boundary(const BWork* work, int n, InstDesc* const* descs, int par, long long* counter,
                     cudaStream_t s) {
    if (n <= 0) return;
    k_boundary<R><<<n, 128, 0, s>>>(work, descs, par, counter);
}

int grid_for(long long nn) {
    long long g = (nn + 255) / 256;
    return (int)std::max<long long>(1, std::min<long long>(g, 152 * 8));
}

lbm_status check_launch() {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(LBM_ECUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
    return LBM_OK;
}

lbm_status status_bits(lbm_ctx* c, unsigned int st) {
    if (st & 4u) {
        c->sticky = LBM_ECUDA;
        return fail(LBM_ECUDA, "dynamic shared memory of the fused kernel is not 128-byte aligned");
    }
    if (st & 2u) {
        c->sticky = LBM_ETIMEOUT;
        return fail(LBM_ETIMEOUT, "a bounded wait on a bulk copy gave up");
    }
    if (st & 1u) {
        c->sticky = LBM_EUNSTABLE;
        return fail(LBM_EUNSTABLE, "non-finite density or temperature detected");
    }
    return LBM_OK;
}

lbm_status read_status(lbm_ctx* c) {
    unsigned int st = 0;
    CUDA_TRY(cudaMemcpyAsync(&st, c->d_status, sizeof(st), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    return status_bits(c, st);
}

bool is_fp32(const lbm_ctx* c) { return c->cfg.precision == LBM_FP32_DEV; }

int cur_buf(const lbm_ctx* c) { return (int)(c->steps & 1); }

}  // namespace

extern "C" {

const char* lbm_last_error(void) { return g_err.c_str(); }

lbm_status lbm_workspace_bytes(const lbm_config* cfg, size_t* bytes) {
    lbm_status st = validate(cfg);
    if (st != LBM_OK) return st;
    if (!bytes) return fail(LBM_EINVAL, "null bytes");
    *bytes = layout_for(*cfg).total;
    return LBM_OK;
}

lbm_status lbm_create(const lbm_config* cfg, void* workspace, size_t workspace_bytes, void* cuda_stream,
                      lbm_ctx** out) {
    if (!out) return fail(LBM_EINVAL, "null out");
    *out = nullptr;
    lbm_status st = validate(cfg);
    if (st != LBM_OK) return st;
    if ((st = configure_kernels()) != LBM_OK) return st;
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    lbm_ctx* c = new lbm_ctx();
    c->cfg = *cfg;
    c->device = dev;
    c->stream = (cudaStream_t)cuda_stream;
    c->L = layout_for(*cfg);
    if (workspace) {
        if (workspace_bytes < c->L.total || ((uintptr_t)workspace & 255u)) {
            delete c;
            return fail(LBM_ENOMEM, "workspace too small or not 256-byte aligned");
        }
        c->ws = (char*)workspace;
        c->ws_bytes = workspace_bytes;
    } else {
        cudaError_t e = cudaMalloc(&c->ws, c->L.total);
        if (e != cudaSuccess) {
            delete c;
            return fail(LBM_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
        }
        c->own_ws = true;
        c->ws_bytes = c->L.total;
    }
    c->d_desc = (InstDesc*)(c->ws + c->L.off_desc);
    c->d_descs = (InstDesc**)(c->ws + c->L.off_descs);
    c->d_status = (unsigned int*)(c->ws + c->L.off_status);
    c->d_counter = (long long*)(c->ws + c->L.off_status + 128);
    c->d_diag = (double*)(c->ws + c->L.off_diag);
    c->d_partials = (double*)(c->ws + c->L.off_partials);
    c->d_snap = (double*)(c->ws + c->L.off_snap);
    c->d_stage = (double*)(c->ws + c->L.off_stage);

    InstDesc& h = c->h;
    h.buf[0] = c->ws + c->L.off_bufA;
    h.buf[1] = c->ws + c->L.off_bufB;
    if ((st = encode_windows(c)) != LBM_OK) {
        lbm_destroy(c);
        return st;
    }
    h.plane = c->L.plane;
    h.nx = cfg->nx;
    h.ny = cfg->ny;
    h.pitch = c->L.pitch;
    h.px = cfg->wall[LBM_WALL_W].periodic != 0;
    h.py = cfg->wall[LBM_WALL_S].periodic != 0;
    h.precision = cfg->precision;
    h.status = c->d_status;
    for (int s = 0; s < 4; ++s) {
        h.wall[s].u[0] = cfg->wall[s].u[0];
        h.wall[s].u[1] = cfg->wall[s].u[1];
        h.wall[s].T = cfg->wall[s].T;
        h.wall[s].thermal = cfg->wall[s].thermal;
        h.wall[s].order = cfg->wall[s].extrap_order;
    }
    auto cleanup = [&](lbm_status s) {
        lbm_destroy(c);
        return s;
    };
    if (cudaMemsetAsync(c->d_status, 0, 256, c->stream) != cudaSuccess) return cleanup(fail(LBM_ECUDA, "memset"));
    InstDesc* p = c->d_desc;
    if (cudaMemcpyAsync(c->d_descs, &p, sizeof(p), cudaMemcpyHostToDevice, c->stream) != cudaSuccess)
        return cleanup(fail(LBM_ECUDA, "descs upload"));
    default_shape(*cfg, lbm::MODEL_ANY, c->bx, c->pair);
    c->by = default_rows(*cfg, c->pair);
    if ((st = upload_work(c)) != LBM_OK) return cleanup(st);
    c->h_bwork = make_bwork(*cfg, 0, 0);
    ensure_tick(c->h_bwork, 0, 0);
    c->n_bwork = (int)c->h_bwork.size();
    if (c->n_bwork) {
        if (cudaMalloc(&c->d_bwork, c->h_bwork.size() * sizeof(BWork)) != cudaSuccess)
            return cleanup(fail(LBM_ENOMEM, "cudaMalloc wall table"));
        if (cudaMemcpyAsync(c->d_bwork, c->h_bwork.data(), c->h_bwork.size() * sizeof(BWork),
                            cudaMemcpyHostToDevice, c->stream) != cudaSuccess)
            return cleanup(fail(LBM_ECUDA, "wall table upload"));
    }
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return cleanup(fail(LBM_ECUDA, "sync"));
    *out = c;
    return LBM_OK;
}

lbm_status lbm_destroy(lbm_ctx* c) {
    if (!c) return LBM_OK;
    if (c->stream) cudaStreamSynchronize(c->stream);
    else cudaDeviceSynchronize();
    if (c->d_work) cudaFree(c->d_work);
    if (c->d_bwork) cudaFree(c->d_bwork);
    if (c->own_ws && c->ws) cudaFree(c->ws);
    delete c;
    return LBM_OK;
}

lbm_status lbm_set_eos(lbm_ctx* c, int kind, const double* params, int np) {
    if (!c) return fail(LBM_EINVAL, "null ctx");
    if (kind < 0 || kind > 3) return fail(LBM_EINVAL, "bad EOS kind");
    const lbm_config& k = c->cfg;
    Params<double> P{};
    double a = 0.0, b = 0.0;
    if (kind == LBM_EOS_CS) b = (np >= 1 && params) ? params[0] : std::sqrt(2.0) * M_PI / (3.0 * k.rho0);
    if (kind == LBM_EOS_CUBIC) {
        if (np < 2 || !params) return fail(LBM_EINVAL, "cubic EOS needs {a, b}");
        a = params[0];
        b = params[1];
        if (!(b * k.rho0 < 1.0)) return fail(LBM_EINVAL, "cubic EOS needs b rho0 < 1");
    }
    // R from dp/drho = c_s^2 = 1/3 at (rho0, T0), Eq. (cs)
    const double cs2 = 1.0 / 3.0, r0 = k.rho0, T0 = k.T0;
    double Rg, p0;
    switch (kind) {
    case LBM_EOS_DECOUPLING:
    case LBM_EOS_IDEAL:
        Rg = cs2 / T0;
        p0 = r0 * Rg * T0;
        break;
    case LBM_EOS_CS: {
        const double e = b * r0 / 4.0;
        const double om = 1.0 - e;
        // d(rho Z)/d rho = (1 + 4e + 4e^2 - 4e^3 + e^4) / (1 - e)^4
        const double dphi = (1.0 + 4.0 * e + 4.0 * e * e - 4.0 * e * e * e + e * e * e * e) / (om * om * om * om);
        Rg = cs2 / (dphi * T0);
        const double Z = (1.0 + e + e * e - e * e * e) / (om * om * om);
        p0 = Z * r0 * Rg * T0;
        break;
    }
    default: {
        const double om = 1.0 - b * r0;
        Rg = (cs2 + 2.0 * a * r0) * om * om / T0;
        p0 = r0 * Rg * T0 / om - a * r0 * r0;
        break;
    }
    }
    if (!(Rg > 0)) return fail(LBM_EINVAL, "EOS gives a non-positive gas constant");
    const double Cv = (p0 / (r0 * T0)) / (k.gamma - 1.0);
    const double Cp = k.gamma * Cv;
    const double w = k.varpi;
    P.rho0 = r0;
    P.T0 = T0;
    P.Cv = Cv;
    P.inv_Cv = 1.0 / Cv;
    P.E0 = Cv * T0;
    P.Rg = Rg;
    P.eos_a = a;
    P.eos_b = b;
    P.p0 = p0;
    P.rho0E0_p0 = r0 * P.E0 + p0;
    P.rho0Cp0 = r0 * Cp;
    P.mu0 = r0 * (k.tau0 - 0.5) * cs2;
    P.inv_T0 = 1.0 / T0;
    P.visc_S = k.visc_p[0];
    P.lam_fac = Cp / k.Pr;
    const double coef = 2.0 / 3.0 + k.gamma1 / 2.0 + k.gamma2 / 3.0;
    if (!(coef > 0)) return fail(LBM_EINVAL, "gamma1, gamma2 give a non-positive conductivity factor");
    P.tj_fac = 1.0 / (coef * r0 * Cp);
    P.e_fac = 3.0 * k.bulk_ratio / w;
    P.alpha1 = -1.0;
    P.beta1 = 1.0;
    P.alpha2 = -(2.0 * P.alpha1 + w + 1.0) / (1.0 - w);
    P.beta2 = -2.0 * P.beta1 / (1.0 - w);
    P.kk = 1.0 - w;
    P.hh = 6.0 * w * (1.0 - w) / (1.0 - 3.0 * w);
    P.bb = (1.0 - w) / (1.0 - 3.0 * w);
    P.gamma1 = k.gamma1;
    P.gamma2 = k.gamma2;
    P.cR11 = -(9.0 - 15.0 * P.kk - 2.0 * P.hh) / (4.0 * w);
    P.cR17 = -3.0 * (9.0 - 3.0 * P.kk + 2.0 * P.hh) / 4.0;
    P.cR18 = 12.0 * (3.0 * P.kk + P.hh);
    P.cR71 = -(3.0 - 4.0 * P.bb) / (4.0 * w);
    P.cR77 = -3.0 * (3.0 + 4.0 * P.bb) / 4.0;
    P.cR81 = P.bb / w;
    P.cR88 = 6.0 * P.bb;
    P.Fx = k.force[0];
    P.Fy = k.force[1];
    P.cs_b0 = 1.0 - b * r0;
    P.dither = c->round_mode == LBM_ROUND_NEAREST ? 0.0 : 1.0;
    P.eos = kind;
    P.visc = k.visc_law;
    P.force_mode = k.force_mode;
    P.corrections = k.corrections;
    c->mc = (k.visc_law == 2 && k.force_mode == 1 && k.corrections && k.force[0] == 0.0 &&
             (kind == lbm::EOS_IDEAL || kind == lbm::EOS_CUBIC) && (long long)k.nx * k.ny >= kModelMinNodes)
                ? lbm::MODEL_CAVITY
                : lbm::MODEL_ANY;
    c->h.pd = P;
    convert_params(P, c->h.pf);
    if (!c->tile_set) {
        // the default shape depends on the model class
        int bx = 0, pair = 0;
        default_shape(k, c->mc, bx, pair);
        if (bx != c->bx || pair != c->pair) {
            c->bx = bx;
            c->pair = pair;
            c->by = default_rows(k, pair);
            lbm_status st = upload_work(c);
            if (st != LBM_OK) return st;
        }
    }

    const double eta0 = (p0 / cs2 - (2.0 + P.alpha1) * r0) / P.beta1;
    const double mr[9] = {r0, 2.0 * P.alpha1 * r0 + 2.0 * P.beta1 * eta0, P.alpha2 * r0 + P.beta2 * eta0, 0, 0, 0, 0, 0, 0};
    const double re = r0 * P.E0, rc = r0 * Cp * T0;
    const double nr[9] = {re, -4.0 * (re - rc) + k.gamma1 * rc, 4.0 * (re - rc) + k.gamma2 * rc, 0, 0, 0, 0, 0, 0};
    host_inverse_moments(mr, c->f_rest);
    host_inverse_moments(nr, c->g_rest);
    c->derived[0] = Rg;
    c->derived[1] = Cv;
    c->derived[2] = Cp;
    c->derived[3] = P.mu0;
    c->derived[4] = p0;
    c->derived[5] = eta0;
    c->derived[6] = Cp * P.mu0 / k.Pr;
    c->derived[7] = cs2;

    CUDA_TRY(cudaMemcpyAsync(c->d_desc, &c->h, sizeof(InstDesc), cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(cudaMemsetAsync(c->d_status, 0, 256, c->stream));
    c->steps = 0;
    c->have_snap = false;
    c->sticky = LBM_OK;
    const long long nn = (long long)k.nx * k.ny;
    if (is_fp32(c)) k_init_rest<float><<<grid_for(nn), 256, 0, c->stream>>>(c->d_desc, 0);
    else k_init_rest<double><<<grid_for(nn), 256, 0, c->stream>>>(c->d_desc, 0);
    lbm_status st = check_launch();
    if (st != LBM_OK) return st;
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    c->eos_set = true;
    return LBM_OK;
}

lbm_status lbm_derived(const lbm_ctx* c, double* out8) {
    if (!c || !out8 || !c->eos_set) return fail(LBM_EINVAL, "context not initialised");
    memcpy(out8, c->derived, sizeof(c->derived));
    return LBM_OK;
}

lbm_status lbm_wait_selftest(lbm_ctx* c, long long limit_cycles) {
    if (!c || !c->eos_set) return fail(LBM_EINVAL, "context not initialised");
    if (limit_cycles < 0 || limit_cycles > (1LL << 32)) return fail(LBM_EINVAL, "limit_cycles must lie in [0, 2^32]");
    k_wait_selftest<<<1, 32, 0, c->stream>>>(c->d_status, limit_cycles);
    lbm_status st = check_launch();
    if (st != LBM_OK) return st;
    return read_status(c);
}

lbm_status lbm_peak_rates(void* cuda_stream, double* out3) {
    if (!out3) return fail(LBM_EINVAL, "null output");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int dev = 0, sms = 152;
    CUDA_TRY(cudaGetDevice(&dev));
    CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = sms * 8, threads = 256;
    void* buf = nullptr;
    CUDA_TRY(cudaMalloc(&buf, (size_t)blocks * threads * sizeof(double)));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    auto cleanup = [&]() {
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        cudaFree(buf);
    };
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cleanup();
        return fail(LBM_ECUDA, "cudaEventCreate");
    }
    const double ops = (double)blocks * threads * kProbeIters * kProbeChains;
    for (int k = 0; k < 3; ++k) {
        float best = 1e30f;
        for (int rep = 0; rep < 3; ++rep) {
            cudaEventRecord(e0, st);
            if (k == 0) k_probe_fp64<<<blocks, threads, 0, st>>>((double*)buf);
            else if (k == 1) k_probe_fp32<<<blocks, threads, 0, st>>>((float*)buf);
            else k_probe_ff64<<<blocks, threads, 0, st>>>((float*)buf);
            cudaEventRecord(e1, st);
            if (cudaEventSynchronize(e1) != cudaSuccess) {
                cleanup();
                return fail(LBM_ECUDA, "probe kernel");
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            best = std::min(best, ms);
        }
        out3[k] = ops / (best * 1e-3);
    }
    cleanup();
    return check_launch();
}

lbm_status lbm_set_rounding(lbm_ctx* c, int mode) {
    if (!c) return fail(LBM_EINVAL, "null ctx");
    if (mode != LBM_ROUND_STOCHASTIC && mode != LBM_ROUND_NEAREST) return fail(LBM_EINVAL, "bad rounding mode");
    c->round_mode = mode;
    const double d = mode == LBM_ROUND_NEAREST ? 0.0 : 1.0;
    c->h.pd.dither = d;
    c->h.pf.dither = (float)d;
    if (c->eos_set)
        CUDA_TRY(cudaMemcpyAsync(c->d_desc, &c->h, sizeof(InstDesc), cudaMemcpyHostToDevice, c->stream));
    return LBM_OK;
}

lbm_status lbm_copy_state(lbm_ctx* d, const lbm_ctx* s) {
    if (!d || !s || !d->eos_set || !s->eos_set) return fail(LBM_EINVAL, "contexts not initialised");
    if (d == s) return LBM_OK;
    lbm_config a = d->cfg, b = s->cfg;
    a.precision = b.precision = 0;
    for (int k = 0; k < 4; ++k) a.wall[k].reserved = b.wall[k].reserved = 0;
    if (memcmp(&a, &b, sizeof(a)) != 0) return fail(LBM_EINVAL, "lbm_copy_state needs the same problem in both contexts");
    if (memcmp(d->f_rest, s->f_rest, sizeof(d->f_rest)) != 0 || memcmp(d->g_rest, s->g_rest, sizeof(d->g_rest)) != 0 ||
        d->h.pd.eos != s->h.pd.eos || d->h.pd.eos_a != s->h.pd.eos_a || d->h.pd.eos_b != s->h.pd.eos_b)
        return fail(LBM_EINVAL, "lbm_copy_state needs the same EOS in both contexts");
    if (s->sticky != LBM_OK) return fail(s->sticky, "source context is unstable");
    CUDA_TRY(cudaStreamSynchronize(s->stream));
    const int nx = s->cfg.nx, ny = s->cfg.ny;
    const long long nn = (long long)nx * ny;
    const int sb = cur_buf(s), db = (int)(s->steps & 1);
    const bool sf = is_fp32(s), df = is_fp32(d);
    void* sp = s->h.buf[sb];
    void* dp = d->h.buf[db];
    const int grid = grid_for(18 * nn);
    if (sf && df) k_copy_state<float, float><<<grid, 256, 0, d->stream>>>((const float*)sp, s->L.plane, s->L.pitch, (float*)dp, d->L.plane, d->L.pitch, nx, ny);
    else if (sf) k_copy_state<float, double><<<grid, 256, 0, d->stream>>>((const float*)sp, s->L.plane, s->L.pitch, (double*)dp, d->L.plane, d->L.pitch, nx, ny);
    else if (df) k_copy_state<double, float><<<grid, 256, 0, d->stream>>>((const double*)sp, s->L.plane, s->L.pitch, (float*)dp, d->L.plane, d->L.pitch, nx, ny);
    else k_copy_state<double, double><<<grid, 256, 0, d->stream>>>((const double*)sp, s->L.plane, s->L.pitch, (double*)dp, d->L.plane, d->L.pitch, nx, ny);
    lbm_status st = check_launch();
    if (st != LBM_OK) return st;
    if (s->have_snap) CUDA_TRY(cudaMemcpyAsync(d->d_snap, s->d_snap, 3 * nn * sizeof(double), cudaMemcpyDeviceToDevice, d->stream));
    CUDA_TRY(cudaMemsetAsync(d->d_status, 0, 256, d->stream));
    CUDA_TRY(cudaStreamSynchronize(d->stream));
    d->steps = s->steps;
    d->have_snap = s->have_snap;
    d->sticky = LBM_OK;
    return LBM_OK;
}

lbm_status lbm_set_tile(lbm_ctx* c, int bx, int by, int pair) {
    if (!c) return fail(LBM_EINVAL, "null ctx");
    if (bx == 0 && by == 0 && pair == 0) {
        // back to the default shape of lbm_create / lbm_set_eos
        default_shape(c->cfg, c->mc, c->bx, c->pair);
        c->by = default_rows(c->cfg, c->pair);
        c->tile_set = false;
        lbm_status st = upload_work(c);
        if (st != LBM_OK) return st;
        CUDA_TRY(cudaStreamSynchronize(c->stream));
        return LBM_OK;
    }
    if (pair != 0 && pair != 4 && c->cfg.precision != LBM_FP32_DEV)
        return fail(LBM_EINVAL, "pair 1-3 and 5 need FP32 storage");
    if (variant_index(bx, pair) < 0)
        return fail(LBM_EINVAL, pair == 4   ? "warp strips (pair 4) are 30, 60 or 120 columns"
                                : pair == 5 ? "paired warp strips (pair 5) are 60, 120 or 240 columns"
                                : (pair == 1 || pair == 2) ? "paired strips (pair 1 or 2) are 64, 128 or 256 columns"
                                                           : "bx must be 32, 64 or 128");
    if (by < 1) return fail(LBM_EINVAL, "by must be >= 1");
    c->bx = bx;
    c->pair = pair;
    c->by = std::min(by, c->cfg.ny);
    c->tile_set = true;
    lbm_status st = upload_work(c);
    if (st != LBM_OK) return st;
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    return LBM_OK;
}

lbm_status lbm_get_tile(const lbm_ctx* c, int* bx, int* by, int* pair) {
    if (!c || !bx || !by || !pair) return fail(LBM_EINVAL, "null argument");
    *bx = c->bx;
    *by = c->by;
    *pair = c->pair;
    return LBM_OK;
}

long lbm_step_count(const lbm_ctx* c) { return c ? c->steps : -1; }

lbm_status lbm_step(lbm_ctx* c, long nsteps) {
    if (!c || !c->eos_set) return fail(LBM_EINVAL, "context not initialised");
    if (nsteps < 0) return fail(LBM_EINVAL, "nsteps < 0");
    if (c->sticky != LBM_OK) return fail(c->sticky, "context is unstable");
    if (nsteps == 0) return LBM_OK;
    const long long base = c->steps;
    CUDA_TRY(cudaMemcpyAsync(c->d_counter, &base, sizeof(base), cudaMemcpyHostToDevice, c->stream));
    for (long s = 0; s < nsteps; ++s) {
        const int par = (int)((c->steps + s) & 1);
        if (is_fp32(c)) {
            launch_collide<float>(c->d_work, c->n_work, variant_index(c->bx, c->pair), c->mc, c->d_descs, par, c->d_counter, c->stream);
            launch_boundary<float>(c->d_bwork, c->n_bwork, c->d_descs, par, c->d_counter, c->stream);
        } else {
            launch_collide<double>(c->d_work, c->n_work, variant_index(c->bx, c->pair), c->mc, c->d_descs, par, c->d_counter, c->stream);
            launch_boundary<double>(c->d_bwork, c->n_bwork, c->d_descs, par, c->d_counter, c->stream);
        }
    }
    lbm_status st = check_launch();
    c->steps += nsteps;
    return st;
}

lbm_status lbm_sync(lbm_ctx* c) {
    if (!c) return fail(LBM_EINVAL, "null ctx");
    if (c->sticky != LBM_OK) return fail(c->sticky, "context is unstable");
    return read_status(c);
}

lbm_status lbm_macros_device(lbm_ctx* c, double* rho, double* ux, double* uy, double* T, double* p) {
    if (!c || !c->eos_set) return fail(LBM_EINVAL, "context not initialised");
    const long long nn = (long long)c->cfg.nx * c->cfg.ny;
    if (is_fp32(c)) k_macros<float><<<grid_for(nn), 256, 0, c->stream>>>(c->d_desc, cur_buf(c), rho, ux, uy, T, p);
    else k_macros<double><<<grid_for(nn), 256, 0, c->stream>>>(c->d_desc, cur_buf(c), rho, ux, uy, T, p);
    return check_launch();
}

lbm_status lbm_macros(lbm_ctx* c, double* rho, double* ux, double* uy, double* T, double* p) {
    if (!c || !c->eos_set) return fail(LBM_EINVAL, "context not initialised");
    const long long nn = (long long)c->cfg.nx * c->cfg.ny;
    double* host[5] = {rho, ux, uy, T, p};
    double* dev[5];
    for (int i = 0; i < 5; ++i) dev[i] = host[i] ? c->d_stage + i * nn : nullptr;
    lbm_status st = lbm_macros_device(c, dev[0], dev[1], dev[2], dev[3], dev[4]);
    if (st != LBM_OK) return st;
    for (int i = 0; i < 5; ++i)
        if (host[i]) CUDA_TRY(cudaMemcpyAsync(host[i], dev[i], nn * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    st = read_status(c);
    if (st != LBM_OK) return st;
    return c->sticky;
}

lbm_status lbm_get_state(lbm_ctx* c, double* f, double* g) {
    if (!c || !c->eos_set) return fail(LBM_EINVAL, "context not initialised");
    const long long nn = (long long)c->cfg.nx * c->cfg.ny;
    for (int q = 0; q < 18; ++q) {
        double* host = q < 9 ? (f ? f + q * nn : nullptr) : (g ? g + (q - 9) * nn : nullptr);
        if (!host) continue;
        const double rest = q < 9 ? c->f_rest[q] : c->g_rest[q - 9];
        if (is_fp32(c)) k_get_plane<float><<<grid_for(nn), 256, 0, c->stream>>>(c->d_desc, cur_buf(c), q, rest, c->d_stage);
        else k_get_plane<double><<<grid_for(nn), 256, 0, c->stream>>>(c->d_desc, cur_buf(c), q, rest, c->d_stage);
        lbm_status st = check_launch();
        if (st != LBM_OK) return st;
        CUDA_TRY(cudaMemcpyAsync(host, c->d_stage, nn * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        CUDA_TRY(cudaStreamSynchronize(c->stream));
    }
    return LBM_OK;
}

lbm_status lbm_set_state(lbm_ctx* c, const double* f, const double* g) {
    if (!c || !c->eos_set || !f || !g) return fail(LBM_EINVAL, "context not initialised or null state");
    const long long nn = (long long)c->cfg.nx * c->cfg.ny;
    for (int q = 0; q < 18; ++q) {
        const double* host = q < 9 ? f + q * nn : g + (q - 9) * nn;
        const double rest = q < 9 ? c->f_rest[q] : c->g_rest[q - 9];
        CUDA_TRY(cudaMemcpyAsync(c->d_stage, host, nn * sizeof(double), cudaMemcpyHostToDevice, c->stream));
        if (is_fp32(c)) k_set_plane<float><<<grid_for(nn), 256, 0, c->stream>>>(c->d_desc, cur_buf(c), q, rest, c->d_stage);
        else k_set_plane<double><<<grid_for(nn), 256, 0, c->stream>>>(c->d_desc, cur_buf(c), q, rest, c->d_stage);
        lbm_status st = check_launch();
        if (st != LBM_OK) return st;
        CUDA_TRY(cudaStreamSynchronize(c->stream));
    }
    CUDA_TRY(cudaMemsetAsync(c->d_status, 0, 256, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    c->sticky = LBM_OK;
    c->have_snap = false;
    return LBM_OK;
}

lbm_status lbm_init_macros(lbm_ctx* c, const double* rho, const double* ux, const double* uy, const double* T) {
    if (!c || !c->eos_set || !rho || !ux || !uy || !T) return fail(LBM_EINVAL, "context not initialised or null field");
    const long long nn = (long long)c->cfg.nx * c->cfg.ny;
    const double* in[4] = {rho, ux, uy, T};
    for (int i = 0; i < 4; ++i)
        CUDA_TRY(cudaMemcpyAsync(c->d_stage + i * nn, in[i], nn * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    if (is_fp32(c))
        k_init_macros<float><<<grid_for(nn), 256, 0, c->stream>>>(c->d_desc, cur_buf(c), c->d_stage, c->d_stage + nn,
                                                                 c->d_stage + 2 * nn, c->d_stage + 3 * nn);
    else
        k_init_macros<double><<<grid_for(nn), 256, 0, c->stream>>>(c->d_desc, cur_buf(c), c->d_stage, c->d_stage + nn,
                                                                  c->d_stage + 2 * nn, c->d_stage + 3 * nn);
    lbm_status st = check_launch();
    if (st != LBM_OK) return st;
    CUDA_TRY(cudaMemsetAsync(c->d_status, 0, 256, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    c->sticky = LBM_OK;
    c->have_snap = false;
    return LBM_OK;
}

lbm_status lbm_nusselt(lbm_ctx* c, int wall, double* nu) {
    if (!c || !c->eos_set || !nu || wall < 0 || wall > 3) return fail(LBM_EINVAL, "bad arguments");
    const lbm_config& k = c->cfg;
    if (k.wall[wall].periodic) return fail(LBM_EINVAL, "periodic side has no wall");
    double tmax = -1e300, tmin = 1e300;
    int nd = 0;
    for (int s = 0; s < 4; ++s)
        if (!k.wall[s].periodic && k.wall[s].thermal == 0) {
            ++nd;
            tmax = std::max(tmax, k.wall[s].T);
            tmin = std::min(tmin, k.wall[s].T);
        }
    if (nd < 2 || !(tmax > tmin)) return fail(LBM_EINVAL, "Nusselt number needs two Dirichlet walls at different T");
    if (is_fp32(c)) k_nusselt<float><<<1, 1024, 0, c->stream>>>(c->d_desc, cur_buf(c), wall, tmax - tmin, c->d_diag + 12);
    else k_nusselt<double><<<1, 1024, 0, c->stream>>>(c->d_desc, cur_buf(c), wall, tmax - tmin, c->d_diag + 12);
    lbm_status st = check_launch();
    if (st != LBM_OK) return st;
    CUDA_TRY(cudaMemcpyAsync(nu, c->d_diag + 12, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    return read_status(c);
}

// The eight outputs of lbm_diagnostics from the FP64 sums of k_diag_final;
// records the new snapshot and turns the context sticky on non-finite nodes.
static lbm_status diag_outputs(lbm_ctx* c, const double* acc, int snapshot, int have, double* out8) {
    const double nn = (double)c->cfg.nx * c->cfg.ny;
    const Params<double>& P = c->h.pd;
    out8[0] = nn * P.rho0 + acc[0];
    out8[1] = nn * P.rho0 * P.E0 + acc[1];
    out8[2] = acc[2];
    double r = 0.0;
    if (have) {
        const double ru = acc[4] > 0 ? std::sqrt(acc[3] / acc[4]) : 0.0;
        const double rT = acc[6] > 0 ? std::sqrt(acc[5] / acc[6]) : 0.0;
        r = std::max(ru, rT);
    }
    out8[3] = r;
    out8[4] = acc[7];
    out8[5] = acc[8];
    out8[6] = acc[9] / nn;
    out8[7] = (double)c->steps;
    if (snapshot) c->have_snap = true;
    if (acc[7] > 0) {
        c->sticky = LBM_EUNSTABLE;
        return fail(LBM_EUNSTABLE, "non-finite nodes in the state");
    }
    return LBM_OK;
}

lbm_status lbm_diagnostics(lbm_ctx* c, int snapshot, double* out8) {
    if (!c || !c->eos_set || !out8) return fail(LBM_EINVAL, "bad arguments");
    const int have = c->have_snap ? 1 : 0;
    if (is_fp32(c))
        k_diag<float><<<kDiagBlocks, kDiagThreads, 0, c->stream>>>(c->d_desc, cur_buf(c), c->d_snap, snapshot, have, c->d_partials);
    else
        k_diag<double><<<kDiagBlocks, kDiagThreads, 0, c->stream>>>(c->d_desc, cur_buf(c), c->d_snap, snapshot, have, c->d_partials);
    k_diag_final<<<1, 32, 0, c->stream>>>(c->d_partials, kDiagBlocks, c->d_diag);
    lbm_status st = check_launch();
    if (st != LBM_OK) return st;
    double acc[kDiagSlots];
    CUDA_TRY(cudaMemcpyAsync(acc, c->d_diag, sizeof(acc), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    st = diag_outputs(c, acc, snapshot, have, out8);
    if (st != LBM_OK) return st;
    return read_status(c);
}

// ------------------------------------------------------------------------
// conserved sums without allocation
// ------------------------------------------------------------------------

// Device address of g_static_partials, looked up once per device.  In host
// code the array's name is only a host-side stand-in, so the kernels are
// given the address that cudaGetSymbolAddress returns for the current device.
static std::mutex g_static_mu;
static double* g_static_addr[64] = {nullptr};

static lbm_status static_scratch(const lbm_ctx* c, double** out) {
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(LBM_EINVAL, "device index out of range");
    // the symbol address is per device: a kernel on the context's stream
    // must get the address on the context's device
    if (dev != c->device)
        return fail(LBM_EINVAL, "the current device (" + std::to_string(dev) + ") is not the context's device (" +
                                    std::to_string(c->device) + "); make the context's device current");
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_partials);
        if (e != cudaSuccess || !p)
            return fail(LBM_ECUDA, std::string("cudaGetSymbolAddress(g_static_partials): ") + cudaGetErrorString(e));
        g_static_addr[dev] = static_cast<double*>(p);
    }
    *out = g_static_addr[dev];
    return LBM_OK;
}

lbm_status lbm_conserved_sums_static(const lbm_ctx* c, double* out4) {
    if (!c || !c->eos_set || !out4) return fail(LBM_EINVAL, "context not initialised or null output");
    const long long nn = (long long)c->cfg.nx * c->cfg.ny;
    const long long nblocks = (nn + kStaticNodesPerBlock - 1) / kStaticNodesPerBlock;
    if (nblocks > kStaticBlocks)
        return fail(LBM_EINVAL, "lbm_conserved_sums_static handles at most " +
                                    std::to_string((long long)kStaticBlocks * kStaticNodesPerBlock) +
                                    " nodes; use lbm_diagnostics for larger lattices");
    double* scratch = nullptr;
    lbm_status st = static_scratch(c, &scratch);
    if (st != LBM_OK) return st;
    // every slot the final pass reads is written first, so nothing needs clearing
    if (is_fp32(c))
        k_sums_static<float><<<(int)nblocks, kStaticThreads, 0, c->stream>>>(c->d_desc, cur_buf(c), scratch);
    else
        k_sums_static<double><<<(int)nblocks, kStaticThreads, 0, c->stream>>>(c->d_desc, cur_buf(c), scratch);
    k_sums_static_final<<<1, 32, 0, c->stream>>>(c->d_desc, scratch, (int)nblocks, out4);
    return check_launch();
}

// ------------------------------------------------------------------------
// batched stepping
// ------------------------------------------------------------------------

static void batch_launch_collide(lbm_batch* b, const LaunchSet& ls, int par, cudaStream_t st) {
    for (int pr = 0; pr < 2; ++pr)
        for (int vi = 0; vi < kVariants; ++vi)
            for (int mc = 0; mc < kModels; ++mc) {
                const int n = ls.w_cnt[pr][vi][mc];
                if (!n) continue;
                const Work* w = b->d_work + ls.w_off[pr][vi][mc];
                if (pr) launch_collide<float>(w, n, vi, mc, b->d_descs, par, ls.counter, st);
                else launch_collide<double>(w, n, vi, mc, b->d_descs, par, ls.counter, st);
            }
}

static void batch_launch_boundary(lbm_batch* b, const LaunchSet& ls, int par, cudaStream_t st) {
    const int last = ls.b_cnt[1] ? 1 : 0;
    for (int pr = 0; pr < 2; ++pr) {
        if (!ls.b_cnt[pr]) continue;
        long long* ctr = (pr == last) ? ls.counter : nullptr;
        if (pr) launch_boundary<float>(b->d_bwork + ls.b_off[pr], ls.b_cnt[pr], b->d_descs, par, ctr, st);
        else launch_boundary<double>(b->d_bwork + ls.b_off[pr], ls.b_cnt[pr], b->d_descs, par, ctr, st);
    }
}

static void batch_launch_step(lbm_batch* b, const LaunchSet& ls, int par, cudaStream_t st) {
    batch_launch_collide(b, ls, par, st);
    batch_launch_boundary(b, ls, par, st);
}

static lbm_status batch_set_counter(lbm_batch* b) {
    const long long v = b->steps;
    CUDA_TRY(cudaMemcpyAsync(b->d_counter, &v, sizeof(v), cudaMemcpyHostToDevice, b->stream));
    return LBM_OK;
}

// Launch groups of the members listed in `members` (indices into ctxs) into
// `ls`, appending their work items to `all` and wall items to `ball`.
static void build_launch_set(lbm_ctx* const* ctxs, const std::vector<int>& members, int shift, LaunchSet& ls,
                             std::vector<Work>& all, std::vector<BWork>& ball) {
    std::vector<Work> groups[2][kVariants][kModels];
    std::vector<BWork> bgroups[2];
    // Members with longer runs first, and each member's runs together in
    // make_work's order (row by row of runs, strips within a row): the
    // CTAs that share a halo row or a 16-byte side chunk then run at about
    // the same time and the second read of it comes from L2.  Sorting the
    // runs themselves by length interleaved the members (their runs differ
    // by a row) and left those re-reads to DRAM.
    auto rows_of = [&](const lbm_ctx* c) {
        return c->tile_set ? c->by : std::max(1, batch_rows(c->cfg, c->pair) >> shift);
    };
    auto run_len = [&](int i) {
        const lbm_config& cf = ctxs[i]->cfg;
        const long long nruns = (cf.ny + rows_of(ctxs[i]) - 1) / rows_of(ctxs[i]);
        return (long long)((cf.ny + nruns - 1) / nruns);
    };
    std::vector<int> order(members);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return run_len(a) > run_len(b); });
    for (int i : order) {
        const lbm_ctx* c = ctxs[i];
        const int pr = is_fp32(c) ? 1 : 0, bi = variant_index(c->bx, c->pair);
        const int par = (int)(c->steps & 1);
        auto w = make_work(c->cfg, i, c->bx, rows_of(c), par, c->steps);
        auto& grp = groups[pr][bi][launch_model(bi, c->mc)];
        grp.insert(grp.end(), w.begin(), w.end());
    }
    for (int i : members) {
        const lbm_ctx* c = ctxs[i];
        auto bw = make_bwork(c->cfg, i, (int)(c->steps & 1));
        bgroups[is_fp32(c) ? 1 : 0].insert(bgroups[is_fp32(c) ? 1 : 0].end(), bw.begin(), bw.end());
    }
    // shorter runs at the end of each launch
    for (int pr = 0; pr < 2; ++pr)
        for (int bi = 0; bi < kVariants; ++bi)
            for (int mc = 0; mc < kModels; ++mc) {
                auto& g = groups[pr][bi][mc];
                if (!g.empty()) split_tail(g, resident_ctas(bi, pr == 1));
                ls.w_off[pr][bi][mc] = (int)all.size();
                ls.w_cnt[pr][bi][mc] = (int)g.size();
                all.insert(all.end(), g.begin(), g.end());
            }
    if (bgroups[0].empty() && bgroups[1].empty()) {
        const lbm_ctx* c = ctxs[members[0]];
        ensure_tick(bgroups[is_fp32(c) ? 1 : 0], members[0], (int)(c->steps & 1));
    }
    for (int pr = 0; pr < 2; ++pr) {
        ls.b_off[pr] = (int)ball.size();
        ls.b_cnt[pr] = (int)bgroups[pr].size();
        ball.insert(ball.end(), bgroups[pr].begin(), bgroups[pr].end());
    }
}

lbm_status lbm_batch_create(lbm_ctx* const* ctxs, int n, int graph_steps, lbm_batch** out) {
    if (!out || !ctxs || n < 1) return fail(LBM_EINVAL, "bad batch arguments");
    *out = nullptr;
    if (graph_steps < 0 || (graph_steps & 1)) return fail(LBM_EINVAL, "graph_steps must be even and >= 0");
    if (!ctxs[0]) return fail(LBM_EINVAL, "null batch member");
    lbm_batch* b = new lbm_batch();
    b->stream = ctxs[0]->stream;
    std::vector<InstDesc*> descs;
    // rows per run of the members whose shape was not set: the batch length,
    // halved for all of them while the batch fills less than the GPU once
    // (each CTA of a member takes 1 / resident_ctas of the GPU)
    int shift = 0;
    for (;; ++shift) {
        double fill = 0.0;
        bool can_halve = false;
        for (int i = 0; i < n; ++i) {
            const lbm_ctx* c = ctxs[i];
            if (!c || c->tile_set) continue;
            const int by = std::max(1, batch_rows(c->cfg, c->pair) >> shift);
            can_halve = can_halve || by > 1;
            fill += (double)cta_count(c->cfg, c->bx, by) /
                    (double)resident_ctas(variant_index(c->bx, c->pair), c->cfg.precision == LBM_FP32_DEV);
        }
        if (fill >= 1.0 || !can_halve) break;
    }
    for (int i = 0; i < n; ++i) {
        lbm_ctx* c = ctxs[i];
        if (!c || !c->eos_set || c->stream != b->stream || c->sticky != LBM_OK) {
            delete b;
            return fail(LBM_EINVAL, "batch members must be initialised, stable and share one stream");
        }
        b->ctxs.push_back(c);
        b->models.push_back(c->mc);
        descs.push_back(c->d_desc);
    }
    std::vector<Work> all;
    std::vector<BWork> ball;
    std::vector<int> everyone(n);
    for (int i = 0; i < n; ++i) everyone[i] = i;
    build_launch_set(ctxs, everyone, shift, b->set, all, ball);
    auto bad = [&](const char* m) {
        lbm_batch_destroy(b);
        return fail(LBM_ECUDA, m);
    };
    if (cudaMalloc(&b->d_descs, descs.size() * sizeof(InstDesc*)) != cudaSuccess) return bad("cudaMalloc descs");
    if (cudaMalloc(&b->d_counter, sizeof(long long)) != cudaSuccess) return bad("cudaMalloc counter");
    if (cudaMemsetAsync(b->d_counter, 0, sizeof(long long), b->stream) != cudaSuccess) return bad("memset counter");
    b->set.counter = b->d_counter;
    if (!all.empty() && cudaMalloc(&b->d_work, all.size() * sizeof(Work)) != cudaSuccess) return bad("cudaMalloc work");
    if (!ball.empty() && cudaMalloc(&b->d_bwork, ball.size() * sizeof(BWork)) != cudaSuccess) return bad("cudaMalloc bwork");
    if (cudaMemcpyAsync(b->d_descs, descs.data(), descs.size() * sizeof(InstDesc*), cudaMemcpyHostToDevice, b->stream) != cudaSuccess)
        return bad("upload descs");
    if (!all.empty() && cudaMemcpyAsync(b->d_work, all.data(), all.size() * sizeof(Work), cudaMemcpyHostToDevice, b->stream) != cudaSuccess)
        return bad("upload work");
    if (!ball.empty() && cudaMemcpyAsync(b->d_bwork, ball.data(), ball.size() * sizeof(BWork), cudaMemcpyHostToDevice, b->stream) != cudaSuccess)
        return bad("upload bwork");
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) return bad("sync");
    b->graph_steps = graph_steps;
    if (graph_steps > 0) {
        if (!b->stream) {
            lbm_batch_destroy(b);
            return fail(LBM_EINVAL, "graph capture needs a non-default stream");
        }
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return bad("begin capture");
        for (int s = 0; s < graph_steps; ++s) batch_launch_step(b, b->set, s & 1, b->stream);
        if (cudaStreamEndCapture(b->stream, &g) != cudaSuccess) return bad("end capture");
        cudaError_t e = cudaGraphInstantiate(&b->graph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return bad("graph instantiate");
    }
    *out = b;
    return LBM_OK;
}

// Rebuild b in place over a new member list: a new batch is built first, so
// b is unchanged when that fails.
static lbm_status batch_rebuild(lbm_batch* b, const std::vector<lbm_ctx*>& members) {
    lbm_batch* nb = nullptr;
    lbm_status st = lbm_batch_create(members.data(), (int)members.size(), b->graph_steps, &nb);
    if (st != LBM_OK) return st;
    lbm_batch old = std::move(*b);
    *b = std::move(*nb);
    *nb = std::move(old);
    return lbm_batch_destroy(nb);
}

lbm_status lbm_batch_add(lbm_batch* b, lbm_ctx* c) {
    if (!b || !c) return fail(LBM_EINVAL, "null batch or context");
    if (std::find(b->ctxs.begin(), b->ctxs.end(), c) != b->ctxs.end()) return fail(LBM_EINVAL, "already a member");
    std::vector<lbm_ctx*> m = b->ctxs;
    m.push_back(c);
    return batch_rebuild(b, m);
}

lbm_status lbm_batch_remove(lbm_batch* b, lbm_ctx* c) {
    if (!b || !c) return fail(LBM_EINVAL, "null batch or context");
    std::vector<lbm_ctx*> m = b->ctxs;
    auto it = std::find(m.begin(), m.end(), c);
    if (it == m.end()) return fail(LBM_EINVAL, "not a member");
    if (m.size() == 1) return fail(LBM_EINVAL, "a batch keeps at least one member; destroy it instead");
    m.erase(it);
    return batch_rebuild(b, m);
}

lbm_status lbm_batch_step(lbm_batch* b, long nsteps) {
    if (!b || nsteps < 0) return fail(LBM_EINVAL, "bad batch step");
    for (size_t i = 0; i < b->ctxs.size(); ++i) {
        if (b->ctxs[i]->sticky != LBM_OK) return fail(b->ctxs[i]->sticky, "a batch member is unstable");
        if (b->ctxs[i]->mc != b->models[i])
            return fail(LBM_EINVAL, "a batch member's EOS class changed since the batch was built; build it again");
    }
    if (nsteps == 0) return LBM_OK;
    lbm_status cs = batch_set_counter(b);
    if (cs != LBM_OK) return cs;
    if (b->graph) {
        if (nsteps % b->graph_steps) return fail(LBM_EINVAL, "nsteps must be a multiple of graph_steps");
        for (long s = 0; s < nsteps; s += b->graph_steps) CUDA_TRY(cudaGraphLaunch(b->graph, b->stream));
    } else {
        for (long s = 0; s < nsteps; ++s) batch_launch_step(b, b->set, (int)((b->steps + s) & 1), b->stream);
        lbm_status st = check_launch();
        if (st != LBM_OK) return st;
    }
    b->steps += nsteps;
    for (lbm_ctx* c : b->ctxs) c->steps += nsteps;
    return LBM_OK;
}

lbm_status lbm_batch_step_profiled(lbm_batch* b, long nsteps, double* ms_collide, double* ms_wall) {
    if (!b || nsteps < 1 || nsteps > 100000 || !ms_collide || !ms_wall) return fail(LBM_EINVAL, "bad profiled step");
    for (size_t i = 0; i < b->ctxs.size(); ++i) {
        if (b->ctxs[i]->sticky != LBM_OK) return fail(b->ctxs[i]->sticky, "a batch member is unstable");
        if (b->ctxs[i]->mc != b->models[i])
            return fail(LBM_EINVAL, "a batch member's EOS class changed since the batch was built; build it again");
    }
    std::vector<cudaEvent_t> ev((size_t)3 * nsteps, nullptr);
    auto cleanup = [&]() {
        for (cudaEvent_t e : ev)
            if (e) cudaEventDestroy(e);
    };
    for (auto& e : ev)
        if (cudaEventCreate(&e) != cudaSuccess) { cleanup(); return fail(LBM_ECUDA, "cudaEventCreate"); }
    lbm_status cs = batch_set_counter(b);
    if (cs != LBM_OK) { cleanup(); return cs; }
    for (long s = 0; s < nsteps; ++s) {
        const int par = (int)((b->steps + s) & 1);
        cudaEventRecord(ev[3 * s], b->stream);
        batch_launch_collide(b, b->set, par, b->stream);
        cudaEventRecord(ev[3 * s + 1], b->stream);
        batch_launch_boundary(b, b->set, par, b->stream);
        cudaEventRecord(ev[3 * s + 2], b->stream);
    }
    lbm_status st = check_launch();
    if (st != LBM_OK) { cleanup(); return st; }
    if (cudaEventSynchronize(ev[3 * nsteps - 1]) != cudaSuccess) { cleanup(); return fail(LBM_ECUDA, "event sync"); }
    double tc = 0.0, tw = 0.0;
    for (long s = 0; s < nsteps; ++s) {
        float a = 0.f, c2 = 0.f;
        cudaEventElapsedTime(&a, ev[3 * s], ev[3 * s + 1]);
        cudaEventElapsedTime(&c2, ev[3 * s + 1], ev[3 * s + 2]);
        tc += a;
        tw += c2;
    }
    cleanup();
    *ms_collide = tc;
    *ms_wall = tw;
    b->steps += nsteps;
    for (lbm_ctx* c : b->ctxs) c->steps += nsteps;
    return LBM_OK;
}

lbm_status lbm_batch_diagnostics(lbm_batch* b, int snapshot, double* out8n, int* member_status) {
    if (!b || !out8n) return fail(LBM_EINVAL, "bad batch diagnostics arguments");
    const int n = (int)b->ctxs.size();
    if (!b->d_jobs) {
        if (cudaMalloc(&b->d_jobs, n * sizeof(DiagJob)) != cudaSuccess ||
            cudaMalloc(&b->d_diag_out, (size_t)n * (kDiagSlots + 1) * sizeof(double)) != cudaSuccess)
            return fail(LBM_ENOMEM, "cudaMalloc batch diagnostics");
        for (int pr = 1; pr >= 0; --pr)
            for (int i = 0; i < n; ++i)
                if ((is_fp32(b->ctxs[i]) ? 1 : 0) == pr) b->diag_order.push_back(i);
    }
    std::vector<DiagJob> jobs(n);
    std::vector<int> have(n);
    int n32 = 0;
    for (int k = 0; k < n; ++k) {
        lbm_ctx* c = b->ctxs[b->diag_order[k]];
        have[k] = c->have_snap ? 1 : 0;
        jobs[k] = DiagJob{c->d_desc, c->d_snap, c->d_partials, c->d_status, cur_buf(c), have[k]};
        n32 += is_fp32(c) ? 1 : 0;
    }
    CUDA_TRY(cudaMemcpyAsync(b->d_jobs, jobs.data(), n * sizeof(DiagJob), cudaMemcpyHostToDevice, b->stream));
    if (n32) k_diag_batch<float><<<dim3(kDiagBlocks, n32), kDiagThreads, 0, b->stream>>>(b->d_jobs, snapshot);
    if (n > n32)
        k_diag_batch<double><<<dim3(kDiagBlocks, n - n32), kDiagThreads, 0, b->stream>>>(b->d_jobs + n32, snapshot);
    k_diag_final_batch<<<n, 32, 0, b->stream>>>(b->d_jobs, kDiagBlocks, b->d_diag_out);
    lbm_status st = check_launch();
    if (st != LBM_OK) return st;
    std::vector<double> acc((size_t)n * (kDiagSlots + 1));
    CUDA_TRY(cudaMemcpyAsync(acc.data(), b->d_diag_out, acc.size() * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
    CUDA_TRY(cudaStreamSynchronize(b->stream));
    for (int k = 0; k < n; ++k) {
        const int i = b->diag_order[k];
        lbm_ctx* c = b->ctxs[i];
        const double* a = acc.data() + (size_t)k * (kDiagSlots + 1);
        lbm_status ms = c->sticky;
        if (ms == LBM_OK) ms = diag_outputs(c, a, snapshot, have[k], out8n + (size_t)i * 8);
        else {
            for (int q = 0; q < 8; ++q) out8n[(size_t)i * 8 + q] = std::nan("");
        }
        if (ms == LBM_OK) ms = status_bits(c, (unsigned int)a[kDiagSlots]);
        if (member_status) member_status[i] = ms;
    }
    return LBM_OK;
}

lbm_status lbm_batch_init_macros(lbm_batch* b, const double* const* rho, const double* const* ux,
                                 const double* const* uy, const double* const* T) {
    if (!b || !rho || !ux || !uy || !T) return fail(LBM_EINVAL, "bad batch init_macros arguments");
    const int n = (int)b->ctxs.size();
    for (int i = 0; i < n; ++i)
        if (!rho[i] || !ux[i] || !uy[i] || !T[i]) return fail(LBM_EINVAL, "null field of batch member " + std::to_string(i));
    // every member's copies and kernels on the shared stream, then one synchronisation
    for (int i = 0; i < n; ++i) {
        lbm_ctx* c = b->ctxs[i];
        const long long nn = (long long)c->cfg.nx * c->cfg.ny;
        const double* in[4] = {rho[i], ux[i], uy[i], T[i]};
        for (int k = 0; k < 4; ++k)
            CUDA_TRY(cudaMemcpyAsync(c->d_stage + k * nn, in[k], nn * sizeof(double), cudaMemcpyHostToDevice, b->stream));
        if (is_fp32(c))
            k_init_macros<float><<<grid_for(nn), 256, 0, b->stream>>>(c->d_desc, cur_buf(c), c->d_stage, c->d_stage + nn,
                                                                     c->d_stage + 2 * nn, c->d_stage + 3 * nn);
        else
            k_init_macros<double><<<grid_for(nn), 256, 0, b->stream>>>(c->d_desc, cur_buf(c), c->d_stage, c->d_stage + nn,
                                                                      c->d_stage + 2 * nn, c->d_stage + 3 * nn);
        lbm_status st = check_launch();
        if (st != LBM_OK) return st;
        CUDA_TRY(cudaMemsetAsync(c->d_status, 0, 256, b->stream));
    }
    CUDA_TRY(cudaStreamSynchronize(b->stream));
    for (lbm_ctx* c : b->ctxs) {
        c->sticky = LBM_OK;
        c->have_snap = false;
    }
    return LBM_OK;
}

lbm_status lbm_batch_macros(lbm_batch* b, double* const* rho, double* const* ux, double* const* uy,
                            double* const* T, double* const* p, int* member_status) {
    if (!b) return fail(LBM_EINVAL, "null batch");
    const int n = (int)b->ctxs.size();
    double* const* fields[5] = {rho, ux, uy, T, p};
    if (!b->d_status_all && cudaMalloc(&b->d_status_all, (size_t)n * sizeof(unsigned int)) != cudaSuccess)
        return fail(LBM_ENOMEM, "cudaMalloc batch status words");
    for (int i = 0; i < n; ++i) {
        lbm_ctx* c = b->ctxs[i];
        const long long nn = (long long)c->cfg.nx * c->cfg.ny;
        double* host[5];
        double* dev[5];
        for (int k = 0; k < 5; ++k) {
            host[k] = fields[k] ? fields[k][i] : nullptr;
            dev[k] = host[k] ? c->d_stage + k * nn : nullptr;
        }
        if (is_fp32(c)) k_macros<float><<<grid_for(nn), 256, 0, b->stream>>>(c->d_desc, cur_buf(c), dev[0], dev[1], dev[2], dev[3], dev[4]);
        else k_macros<double><<<grid_for(nn), 256, 0, b->stream>>>(c->d_desc, cur_buf(c), dev[0], dev[1], dev[2], dev[3], dev[4]);
        lbm_status st = check_launch();
        if (st != LBM_OK) return st;
        for (int k = 0; k < 5; ++k)
            if (host[k]) CUDA_TRY(cudaMemcpyAsync(host[k], dev[k], nn * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
        CUDA_TRY(cudaMemcpyAsync(b->d_status_all + i, c->d_status, sizeof(unsigned int), cudaMemcpyDeviceToDevice, b->stream));
    }
    std::vector<unsigned int> words(n);
    CUDA_TRY(cudaMemcpyAsync(words.data(), b->d_status_all, (size_t)n * sizeof(unsigned int), cudaMemcpyDeviceToHost, b->stream));
    CUDA_TRY(cudaStreamSynchronize(b->stream));
    for (int i = 0; i < n; ++i) {
        lbm_ctx* c = b->ctxs[i];
        lbm_status ms = status_bits(c, words[i]);
        if (ms == LBM_OK) ms = c->sticky;
        if (member_status) member_status[i] = ms;
    }
    return LBM_OK;
}

lbm_status lbm_batch_destroy(lbm_batch* b) {
    if (!b) return LBM_OK;
    if (b->stream) cudaStreamSynchronize(b->stream);
    else cudaDeviceSynchronize();
    if (b->d_jobs) cudaFree(b->d_jobs);
    if (b->d_diag_out) cudaFree(b->d_diag_out);
    if (b->d_status_all) cudaFree(b->d_status_all);
    if (b->graph) cudaGraphExecDestroy(b->graph);
    if (b->d_counter) cudaFree(b->d_counter);
    if (b->d_descs) cudaFree(b->d_descs);
    if (b->d_work) cudaFree(b->d_work);
    if (b->d_bwork) cudaFree(b->d_bwork);
    delete b;
    return LBM_OK;
}

}  // extern "C"
