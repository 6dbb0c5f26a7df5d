// Learned initialisation: 3x3x3 convolution layers (forward, input adjoint,
// weight adjoint) on the 5th-generation tensor cores of sm_103a.
//
// The paper names learning-based registration as planned work (Sec. I,
// Sec. V) without a network. This library trains a small encoder-decoder
// that predicts the B-spline coefficients of a pair. Its layers are dense
// contractions, and they are written here as implicit GEMMs:
//
//   forward   out[o][co]   = sum_{t, ci} in[s o + d_t][ci] * w[co][t][ci]
//             M = output voxels, N = cout, K = 27 cin (k = t cin + ci)
//   dgrad     g_in[p][ci]  = sum_{t, co} g_out[(p - d_t)/s][co] * w[co][t][ci]
//             M = input voxels,  N = cin,  K = (live taps) cout (k = tap cout + co)
//             With stride 2 only the taps whose (p - d_t)/2 is an integer
//             reach p: one per axis where p is even (d = 0), two where it
//             is odd (d = -1, +1). The input voxels are split into the 8
//             parity classes of (z, y, x), and each class runs over its own
//             1 to 8 taps instead of 27.
//   wgrad     g_w[(t,ci)][co] = sum_o in[s o + d_t][ci] * g_out[o][co]
//             M = 27 cin (+1: a row of ones gives the bias gradient),
//             N = cout, K = output voxels (split over blocks, partials
//             summed in a fixed order by k_wgrad_reduce)
//
// Activations are bf16, channels last ([b][z][y][x][c]); accumulation is
// fp32 in tensor memory. A CTA of 4 warps owns a 128-row tile of D in TMEM
// (tcgen05.alloc) and walks a stream of work items (one K slice of 64 of a
// tile each, tile after tile, the CTA's tiles strided by the grid). The
// threads gather the im2col operand of the next item with cp.async
// (16-byte copies, zero-filled at the faces) into a 2-slot shared-memory
// ring (a 3-slot ring two items ahead fitted fewer CTAs per SM and was
// slower: these gathers want resident warps more than depth); the weight
// operand of the forward and dgrad passes is stored pre-tiled in the
// shared-memory layout, so each slice of it arrives
// with one cp.async.bulk on an mbarrier. One thread issues tcgen05.mma
// (kind::f16, bf16 x bf16 -> f32, M = 128, K = 16 per instruction) on
// shared-memory descriptors and a tcgen05.commit frees the slot; after the
// last slice of a tile the threads read D back with tcgen05.ld while the
// next tile's gathers are already in flight.
//
// Shared-memory operand layout (no swizzle): 8 x 8 core matrices of 128 B
// (eight 16-byte rows). For the K-major operands (forward, dgrad) a row is 8
// consecutive K elements of one M/N index; for the MN-major operands (wgrad,
// whose K runs over voxels) a row is 8 consecutive M/N elements at one K
// index, which is exactly one 16-byte channel group of a voxel, so no
// transposition is needed. In both cases the core matrices of a tile are
// placed 128 B apart along K and 1024 B apart along M/N.
//
// Every wait on an mbarrier is bounded (about one second of %globaltimer);
// a wait that runs out records AL_ERR_TIMEOUT in the layer error word and
// the kernel carries on to its end, so no launch can hang.
#include <cuda_bf16.h>
#include <stdint.h>

#include <mutex>

#include "launch.h"
#include "profile.h"

namespace airgb {

namespace {

__device__ int g_conv_error = 0;

constexpr int kThreads = 128;
constexpr int kStages = 2;                    // shared-memory ring slots
constexpr int kAhead = 1;                     // items gathered ahead of the MMA (< kStages)
constexpr int kBK = 64;                       // K elements per ring slot
constexpr int kATile = 128 * kBK * 2;         // bytes of one A slot (16 KB)
// wgrad and split-K blocks aimed at (8 per SM of a 152-SM GB300). A constant,
// not the device's SM count: the split counts size workspaces, which must not
// depend on the device the sizes are queried on.
constexpr int kTargetUnits = 1216;
constexpr int kMaxN = 128;
constexpr int kErrTimeout = 6;                // AL_ERR_TIMEOUT
constexpr int kMaxClasses = 8;

enum { FWD = 0, DGRAD = 1, WGRAD = 2 };

struct ConvArgs {
    const __nv_bfloat16 *act;    // FWD/WGRAD: layer input; DGRAD: grad of the output
    const __nv_bfloat16 *gout;   // WGRAD: grad of the output
    const __nv_bfloat16 *wpk;    // FWD/DGRAD: weight slices in the shared-memory layout
    const float *bias;           // FWD (nullable)
    const __nv_bfloat16 *mask;   // DGRAD: ReLU factor (x_in > 0), N channels (nullable)
    const __nv_bfloat16 *addend; // DGRAD: added before the ReLU factor (nullable)
    void *out;
    int D, H, W, Do, Ho, Wo;     // input and output grid of the layer
    int cin, cout, stride;
    int N;                       // GEMM N
    int Kreal;                   // FWD 27 cin; DGRAD 27 cout (stride 1); WGRAD voxels per split
    int units, mtiles;           // work units (tiles); WGRAD: M tiles (units = mtiles x splits)
    int rows;                    // FWD: output voxels; DGRAD: input voxels; WGRAD: output voxels
    int relu, out_f32, add_stride, add_off;
    int64_t act_elems, gout_elems;  // elements of act and gout (checked builds)
    float *part;                 // FWD with split K: fp32 partials [class][rows][N]
    int classes;                 // DGRAD with stride 2: 8 parity classes; otherwise 1
    int cls_unit0[kMaxClasses + 1];  // first unit of each class; [classes] = units
    int cls_nst[kMaxClasses];        // K slices of a unit of each class
    int cls_slice0[kMaxClasses];     // first packed weight slice of each class
    uint32_t idesc, tmem_cols;
};

// ---- PTX wrappers ----------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t globaltimer()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for the phase of `bar` with this parity to complete, for about one
// second at most; false (and AL_ERR_TIMEOUT recorded) if it did not.
__device__ __noinline__ bool mbar_wait(uint32_t bar, uint32_t parity)
{
    if (mbar_try_wait(bar, parity))
        return true;
    const uint64_t t0 = globaltimer();
    while (!mbar_try_wait(bar, parity)) {
        if (globaltimer() - t0 > 1000000000ull) {
            atomicExch(&g_conv_error, kErrTimeout);
            return false;
        }
    }
    return true;
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_load(uint32_t dst, const void *src, uint32_t bytes,
                                          uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void fence_proxy_async()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t slot, uint32_t cols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot),
                 "r"(cols)
                 : "memory");
}

__device__ __forceinline__ void tmem_relinquish()
{
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t cols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(cols)
                 : "memory");
}

__device__ __forceinline__ void tc_before_sync()
{
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tc_after_sync()
{
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// D[tmem] (+)= A * B^T for one K = 16 slice (bf16 operands, fp32 accumulator).
__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accumulate)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Arrive on `bar` once every tcgen05.mma issued so far by this thread is done.
__device__ __forceinline__ void tc_commit(uint32_t bar)
{
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
        : "memory");
}

// 16 consecutive fp32 columns of this thread's TMEM lane (warp w reads lanes
// 32w .. 32w + 31), waiting for the load to complete.
__device__ __forceinline__ void tc_load16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
        "%11, %12, %13, %14, %15}, [%16];\n"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i)
        v[i] = __uint_as_float(r[i]);
}

// Shared-memory matrix descriptor, no swizzle: start address, the byte
// distance between core matrices along K (leading) and along M/N (stride),
// descriptor version 1 (bits 46-47) of sm_100-class tensor cores.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr)
{
    constexpr uint64_t lbo = 128, sbo = 1024;
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((lbo >> 4) << 16) | ((sbo >> 4) << 32) |
           (1ull << 46);
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&h);
}

__device__ __forceinline__ float bf16_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t w) { return __uint_as_float(w & 0xFFFF0000u); }

// Byte offset of row `r` (M or N index) and 16-byte chunk `kc` in a K-major
// tile, and of K row `k` of the core matrices of M/N group `g` in an
// MN-major tile: both put core matrices 128 B apart along K, 1024 B along M/N.
__device__ __forceinline__ int kmajor_off(int r, int kc) { return (r >> 3) * 1024 + kc * 128 + (r & 7) * 16; }
__device__ __forceinline__ int mnmajor_off(int g, int k) { return g * 1024 + (k >> 3) * 128 + (k & 7) * 16; }


__device__ __forceinline__ void cp16(uint32_t dst, const void *src, bool ok)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src),
                 "r"(ok ? 16 : 0)
                 : "memory");
}

__device__ __forceinline__ void cp4(uint32_t dst, const void *src, bool ok)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(dst), "l"(src),
                 "r"(ok ? 4 : 0)
                 : "memory");
}

__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

template <int N>
__device__ __forceinline__ void cp_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

__device__ __forceinline__ size_t vox_index(int b, int z, int y, int x, int D, int H, int W)
{
    return (((size_t)b * D + z) * H + y) * W + x;
}

// Position of a work item: unit u (a 128-row tile; its class and index in
// the class), slice kk of the unit's nst slices.
struct Cursor {
    int u, kk, cls, tile, nst;
};

__device__ __forceinline__ void cursor_set(Cursor &c, int units, int classes, const int *unit0,
                                           const int *nst)
{
    if (c.u >= units) {
        c.nst = 0;
        return;
    }
    int k = 0;
    while (k + 1 < classes && c.u >= unit0[k + 1])
        ++k;
    c.cls = k;
    c.tile = c.u - unit0[k];
    c.nst = nst[k];
}

// Parity class geometry of the stride-2 dgrad: class bits (z, y, x), the
// number of input voxels of the class per axis, and its taps per axis.
struct ClassGeo {
    int cz, cy, cx, Qz, Qy, Qx, rows;
};

__device__ __forceinline__ ClassGeo class_geo(const ConvArgs &a, int cls)
{
    ClassGeo g;
    g.cz = (cls >> 2) & 1;
    g.cy = (cls >> 1) & 1;
    g.cx = cls & 1;
    g.Qz = (a.D - g.cz + 1) / 2;
    g.Qy = (a.H - g.cy + 1) / 2;
    g.Qx = (a.W - g.cx + 1) / 2;
    g.rows = g.Qz * g.Qy * g.Qx * (a.rows / (a.D * a.H * a.W));
    return g;
}

// ---- operand fills ---------------------------------------------------------
// Tables shared by a CTA (built once per launch, row independent):
//   tapoff[t]      element offset of tap t from the origin of a row's taps:
//                  FWD and WGRAD: input voxel s o - 1 per axis, offset
//                  ((tz H + ty) W + tx) cin; DGRAD stride 1: output voxel
//                  p + 1 per axis, offset -((tz Ho + ty) Wo + tx) cout
//   ctoff[c][ti]   DGRAD stride 2: offset ((az Ho + ay) Wo + ax) cout of
//                  tap index ti of parity class c from output voxel q
struct Tables {
    int tapoff[27];
    int ctoff[kMaxClasses][8];
};

__device__ __forceinline__ void build_tables(const ConvArgs &a, Tables &T, int tid, int mode)
{
    if (tid < 27) {
        const int tz = tid / 9, ty = (tid / 3) % 3, tx = tid % 3;
        T.tapoff[tid] = mode == DGRAD ? -((tz * a.Ho + ty) * a.Wo + tx) * a.cout
                                      : ((tz * a.H + ty) * a.W + tx) * a.cin;
    }
    if (tid < kMaxClasses * 8) {
        const int cls = tid >> 3, ti = tid & 7;
        const int cz = (cls >> 2) & 1, cy = (cls >> 1) & 1, cx = cls & 1;
        const int ix = cx ? (ti & 1) : 0;
        const int iy = cy ? ((ti >> cx) & 1) : 0;
        const int iz = ti >> (cx + cy);
        const int az = cz & (iz == 0), ay = cy & (iy == 0), ax = cx & (ix == 0);
        T.ctoff[cls][ti] = ((az * a.Ho + ay) * a.Wo + ax) * a.cout;
    }
}

// Per-thread state of the unit (tile) the producer is filling.
struct UnitState {
    int64_t rowoff;  // FWD/DGRAD: element offset of the row's tap origin (used only with a valid tap)
    uint32_t mask;   // FWD/DGRAD: valid taps (bit t, or bit ti for a parity class)
    int m0;          // WGRAD: first M row of this thread's 8 groups
    int kreal;       // WGRAD: 27 cin
};

template <int MODE>
__device__ __forceinline__ void unit_begin(const ConvArgs &a, const Cursor &c, int tid,
                                           UnitState &st)
{
    if (MODE == FWD) {
        const int row = c.tile * 128 + tid;
        st.mask = 0;
        st.rowoff = 0;
        if (row < a.rows) {
            int r = row;
            const int ox = r % a.Wo;
            r /= a.Wo;
            const int oy = r % a.Ho;
            r /= a.Ho;
            const int oz = r % a.Do;
            const int b = r / a.Do;
            const int z0 = oz * a.stride - 1, y0 = oy * a.stride - 1, x0 = ox * a.stride - 1;
            st.rowoff = ((((int64_t)b * a.D + z0) * a.H + y0) * a.W + x0) * a.cin;
            uint32_t mz = 0, my = 0, mx = 0;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                mz |= (uint32_t)((unsigned)(z0 + d) < (unsigned)a.D) << d;
                my |= (uint32_t)((unsigned)(y0 + d) < (unsigned)a.H) << d;
                mx |= (uint32_t)((unsigned)(x0 + d) < (unsigned)a.W) << d;
            }
#pragma unroll
            for (int t = 0; t < 27; ++t)
                st.mask |= (((mz >> (t / 9)) & (my >> ((t / 3) % 3)) & (mx >> (t % 3))) & 1u) << t;
        }
    } else if (MODE == DGRAD) {
        st.mask = 0;
        st.rowoff = 0;
        if (a.classes == 1) {
            const int row = c.tile * 128 + tid;
            if (row < a.rows) {
                int r = row;
                const int x = r % a.W;
                r /= a.W;
                const int y = r % a.H;
                r /= a.H;
                const int z = r % a.D;
                const int b = r / a.D;
                // output voxel p - d = p + 1 - t per axis, t in 0..2
                st.rowoff = ((((int64_t)b * a.Do + z + 1) * a.Ho + y + 1) * a.Wo + x + 1) * a.cout;
                uint32_t mz = 0, my = 0, mx = 0;
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    mz |= (uint32_t)((unsigned)(z + 1 - d) < (unsigned)a.Do) << d;
                    my |= (uint32_t)((unsigned)(y + 1 - d) < (unsigned)a.Ho) << d;
                    mx |= (uint32_t)((unsigned)(x + 1 - d) < (unsigned)a.Wo) << d;
                }
#pragma unroll
                for (int t = 0; t < 27; ++t)
                    st.mask |= (((mz >> (t / 9)) & (my >> ((t / 3) % 3)) & (mx >> (t % 3))) & 1u)
                               << t;
            }
        } else {
            const ClassGeo g = class_geo(a, c.cls);
            const int row = c.tile * 128 + tid;
            if (row < g.rows) {
                int r = row;
                const int qx = r % g.Qx;
                r /= g.Qx;
                const int qy = r % g.Qy;
                r /= g.Qy;
                const int qz = r % g.Qz;
                const int b = r / g.Qz;
                st.rowoff = ((((int64_t)b * a.Do + qz) * a.Ho + qy) * a.Wo + qx) * a.cout;
                // adjacency 1 is reachable only when q + 1 is inside
                const uint32_t okz1 = (unsigned)(qz + 1) < (unsigned)a.Do,
                               oky1 = (unsigned)(qy + 1) < (unsigned)a.Ho,
                               okx1 = (unsigned)(qx + 1) < (unsigned)a.Wo;
                const uint32_t okz0 = (unsigned)qz < (unsigned)a.Do,
                               oky0 = (unsigned)qy < (unsigned)a.Ho,
                               okx0 = (unsigned)qx < (unsigned)a.Wo;
                const int ntaps = (1 + g.cz) * (1 + g.cy) * (1 + g.cx);
                for (int ti = 0; ti < ntaps; ++ti) {
                    const int ix = g.cx ? (ti & 1) : 0;
                    const int iy = g.cy ? ((ti >> g.cx) & 1) : 0;
                    const int iz = ti >> (g.cx + g.cy);
                    // odd axis: i = 0 is tap d = -1, reading output q + 1
                    const uint32_t az = g.cz & (iz == 0), ay = g.cy & (iy == 0),
                                   ax = g.cx & (ix == 0);
                    const uint32_t ok = (az ? okz1 : okz0) & (ay ? oky1 : oky0) & (ax ? okx1 : okx0);
                    st.mask |= ok << ti;
                }
            }
        }
    } else {
        const int mt = c.u % a.mtiles;
        st.m0 = mt * 128 + (tid >> 6) * 64;
        st.kreal = 27 * a.cin;
    }
}

// This thread's share of one work item (slot A, B).
template <int MODE>
__device__ __forceinline__ void fill_item(const ConvArgs &a, const Cursor &c, const UnitState &st,
                                          uint8_t *A, uint8_t *B, int tid, const int *tapoff,
                                          const int (*ctoff)[8], int kslice0)
{
    const uint32_t sA = (uint32_t)__cvta_generic_to_shared(A);
    if (MODE == FWD) {
        if (a.cin == 2) {
            // K = 54: word t (2 channels) of tap t; chunk t / 4, word t % 4
            const uint32_t *src = reinterpret_cast<const uint32_t *>(a.act);
#pragma unroll
            for (int t = 0; t < 32; ++t) {
                bool ok = t < 27 && ((st.mask >> (t & 31)) & 1u);
                if (ok && !(al_index_ok(st.rowoff + tapoff[t], a.act_elems - 1)))
                    ok = false;
                cp4(sA + kmajor_off(tid, t >> 2) + (t & 3) * 4,
                    ok ? src + (st.rowoff + tapoff[t < 27 ? t : 0]) / 2 : src, ok);
            }
        } else {
            // with split K the unit's slices start at slice kslice0 of the layer
            int k = (kslice0 + c.kk) * kBK;
            int t = k / a.cin, ci = k - t * a.cin;
#pragma unroll
            for (int kc = 0; kc < 8; ++kc, k += 8) {
                bool ok = k < a.Kreal && ((st.mask >> t) & 1u);
                if (ok && !al_index_ok(st.rowoff + tapoff[t] + ci, a.act_elems - 7))
                    ok = false;
                cp16(sA + kmajor_off(tid, kc),
                     ok ? a.act + st.rowoff + tapoff[ok ? t : 0] + ci : a.act, ok);
                ci += 8;  // next group of 8 channels (cin is a multiple of 8)
                if (ci >= a.cin) {
                    ci -= a.cin;
                    ++t;
                }
            }
        }
    } else if (MODE == DGRAD) {
        const int k0 = c.kk * kBK;
        int t = k0 / a.cout, co = k0 - t * a.cout;
#pragma unroll
        for (int kc = 0; kc < 8; ++kc, co += 8) {
            if (co >= a.cout) {
                co -= a.cout;
                ++t;
            }
            bool ok = t < 27 && ((st.mask >> (t & 31)) & 1u);
            int off = 0;
            if (ok)
                off = a.classes == 1 ? tapoff[t] : ctoff[c.cls][t];
            if (ok && !al_index_ok(st.rowoff + off + co, a.act_elems - 7))
                ok = false;
            cp16(sA + kmajor_off(tid, kc), ok ? a.act + st.rowoff + off + co : a.act, ok);
        }
    } else {
        // A: rows m = (t, ci) of the M tile, K = 64 voxels. Thread tid owns
        // voxel k = tid % 64 of the slice and half h = tid / 64 of the M
        // groups; 8 consecutive lanes write 8 consecutive K rows of one core
        // matrix (128 contiguous bytes).
        const int vbeg = (c.u / a.mtiles) * a.Kreal;
        const int vend = min(vbeg + a.Kreal, a.rows);
        const int k = tid & (kBK - 1), h = tid >> 6;
        const int vox = vbeg + c.kk * kBK + k;
        const bool vok = vox < vend;
        int r = vok ? vox : 0;
        const int ox = r % a.Wo;
        r /= a.Wo;
        const int oy = r % a.Ho;
        r /= a.Ho;
        const int oz = r % a.Do;
        const int bb = r / a.Do;
        const int zz = oz * a.stride - 1, yy = oy * a.stride - 1, xx = ox * a.stride - 1;
        uint32_t mz = 0, my = 0, mx = 0;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            mz |= (uint32_t)((unsigned)(zz + d) < (unsigned)a.D) << d;
            my |= (uint32_t)((unsigned)(yy + d) < (unsigned)a.H) << d;
            mx |= (uint32_t)((unsigned)(xx + d) < (unsigned)a.W) << d;
        }
        if (!vok)
            mz = 0;
        const int64_t org = ((((int64_t)bb * a.D + zz) * a.H + yy) * a.W + xx) * a.cin;
        if (a.cin == 2) {
            // word t of the 55 rows (tap t, 2 channels; t = 27 the bias row),
            // 14 words per thread; words 28..31 and the groups past them stay
            // zero (cleared once: a 2-channel layer has one M tile)
            const uint32_t *src = reinterpret_cast<const uint32_t *>(a.act);
#pragma unroll
            for (int j = 0; j < 14; ++j) {
                const int t = h * 14 + j;
                const int off = mnmajor_off(t >> 2, k) + (t & 3) * 4;
                if (t == 27) {
                    *reinterpret_cast<uint32_t *>(A + off) = vok ? 0x3F80u : 0u;
                } else {
                    bool ok = ((mz >> (t / 9)) & (my >> ((t / 3) % 3)) & (mx >> (t % 3))) & 1u;
                    if (ok && !al_index_ok(org + tapoff[t], a.act_elems - 1))
                        ok = false;
                    cp4(sA + off, ok ? src + (org + tapoff[t]) / 2 : src, ok);
                }
            }
        } else {
            int m0 = st.m0;
            int t = m0 / a.cin, ci = m0 - t * a.cin;
#pragma unroll
            for (int j = 0; j < 8; ++j, m0 += 8) {
                const int g = h * 8 + j;
                const int off = mnmajor_off(g, k);
                if (m0 < st.kreal) {
                    bool ok = ((mz >> (t / 9)) & (my >> ((t / 3) % 3)) & (mx >> (t % 3))) & 1u;
                    if (ok && !al_index_ok(org + tapoff[t] + ci, a.act_elems - 7))
                        ok = false;
                    cp16(sA + off, ok ? a.act + org + tapoff[t] + ci : a.act, ok);
                } else if (m0 == st.kreal) {
                    *reinterpret_cast<uint4 *>(A + off) = make_uint4(vok ? 0x3F80u : 0u, 0, 0, 0);
                } else if (a.mtiles > 1) {
                    *reinterpret_cast<uint4 *>(A + off) = make_uint4(0, 0, 0, 0);
                }
                ci += 8;
                if (ci >= a.cin) {
                    ci -= a.cin;
                    ++t;
                }
            }
        }
        // B: rows n = co (N / 8 groups) x 64 voxels
        const int kbase = vbeg + c.kk * kBK;
        const uint32_t sB = (uint32_t)__cvta_generic_to_shared(B);
        const int ng = a.N >> 3;
        for (int idx = tid; idx < ng * kBK; idx += kThreads) {
            const int krow = idx & 7, cm = idx >> 3;
            const int g = cm % ng, kg = cm / ng;
            const int kk2 = kg * 8 + krow;
            const int v = kbase + kk2;
            bool ok = v < vend;
            if (ok && !al_index_ok((int64_t)v * a.cout + g * 8, a.gout_elems - 7))
                ok = false;
            cp16(sB + mnmajor_off(g, kk2), ok ? a.gout + (size_t)v * a.cout + g * 8 : a.gout, ok);
        }
    }
}

// ---- epilogue: row tid of the finished tile from TMEM lane tid -------------
template <int MODE>
__device__ __forceinline__ void epilogue(const ConvArgs &a, const Cursor &c, uint32_t lane_addr,
                                         int tid)
{
    size_t orow = 0;
    bool valid = true;
    if (MODE == FWD) {
        const int row = c.tile * 128 + tid;
        valid = row < a.rows;
        orow = (size_t)row;
    } else if (MODE == DGRAD) {
        if (a.classes == 1) {
            const int row = c.tile * 128 + tid;
            valid = row < a.rows;
            orow = (size_t)row;
        } else {
            const ClassGeo g = class_geo(a, c.cls);
            const int row = c.tile * 128 + tid;
            valid = row < g.rows;
            int r = valid ? row : 0;
            const int qx = r % g.Qx;
            r /= g.Qx;
            const int qy = r % g.Qy;
            r /= g.Qy;
            const int qz = r % g.Qz;
            const int b = r / g.Qz;
            orow = vox_index(b, 2 * qz + g.cz, 2 * qy + g.cy, 2 * qx + g.cx, a.D, a.H, a.W);
        }
    } else {
        const int mt = c.u % a.mtiles, split = c.u / a.mtiles;
        orow = (size_t)split * a.mtiles * 128 + (size_t)mt * 128 + tid;
    }
    for (int c0 = 0; c0 < a.N; c0 += 16) {
        float v[16];
        tc_load16(lane_addr + (uint32_t)c0, v);
        if (!valid)
            continue;
        if (MODE == FWD && a.part) {
            // split K: this K partition's partial sums, reduced by k_fwd_reduce
            float4 *o = reinterpret_cast<float4 *>(a.part + ((size_t)c.cls * a.rows + orow) * a.N + c0);
#pragma unroll
            for (int q = 0; q < 4; ++q)
                o[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
            continue;
        }
        if (MODE == FWD) {
            if (a.bias) {
#pragma unroll
                for (int i = 0; i < 16; ++i)
                    v[i] += __ldg(a.bias + c0 + i);
            }
            if (a.relu) {
#pragma unroll
                for (int i = 0; i < 16; ++i)
                    v[i] = fmaxf(v[i], 0.0f);
            }
        } else if (MODE == DGRAD) {
            if (a.addend) {
                const uint4 *p = reinterpret_cast<const uint4 *>(a.addend + orow * a.add_stride +
                                                                 a.add_off + c0);
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const uint4 w = __ldg(p + q);
                    const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
                    for (int h = 0; h < 4; ++h) {
                        v[8 * q + 2 * h] += bf16_lo(ws[h]);
                        v[8 * q + 2 * h + 1] += bf16_hi(ws[h]);
                    }
                }
            }
            if (a.mask) {
                const uint4 *p = reinterpret_cast<const uint4 *>(a.mask + orow * a.N + c0);
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const uint4 w = __ldg(p + q);
                    const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
                    for (int h = 0; h < 4; ++h) {
                        if (!(bf16_lo(ws[h]) > 0.0f))
                            v[8 * q + 2 * h] = 0.0f;
                        if (!(bf16_hi(ws[h]) > 0.0f))
                            v[8 * q + 2 * h + 1] = 0.0f;
                    }
                }
            }
        }
        if (MODE == WGRAD || (MODE == FWD && a.out_f32)) {
            float4 *o = reinterpret_cast<float4 *>(static_cast<float *>(a.out) + orow * a.N + c0);
#pragma unroll
            for (int q = 0; q < 4; ++q)
                o[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
        } else {
            uint4 *o = reinterpret_cast<uint4 *>(static_cast<__nv_bfloat16 *>(a.out) + orow * a.N +
                                                 c0);
            o[0] = make_uint4(pack_bf16(v[0], v[1]), pack_bf16(v[2], v[3]), pack_bf16(v[4], v[5]),
                              pack_bf16(v[6], v[7]));
            o[1] = make_uint4(pack_bf16(v[8], v[9]), pack_bf16(v[10], v[11]),
                              pack_bf16(v[12], v[13]), pack_bf16(v[14], v[15]));
        }
    }
}

// Before the last MMAs of a dgrad tile complete: pull this row's ReLU-factor
// and addend channels towards L2, so the epilogue's reads do not wait on DRAM.
__device__ __forceinline__ void dgrad_prefetch(const ConvArgs &a, const Cursor &c, int tid)
{
    size_t orow;
    if (a.classes == 1) {
        const int row = c.tile * 128 + tid;
        if (row >= a.rows)
            return;
        orow = (size_t)row;
    } else {
        const ClassGeo g = class_geo(a, c.cls);
        const int row = c.tile * 128 + tid;
        if (row >= g.rows)
            return;
        int r = row;
        const int qx = r % g.Qx;
        r /= g.Qx;
        const int qy = r % g.Qy;
        r /= g.Qy;
        const int qz = r % g.Qz;
        const int b = r / g.Qz;
        orow = vox_index(b, 2 * qz + g.cz, 2 * qy + g.cy, 2 * qx + g.cx, a.D, a.H, a.W);
    }
    if (a.mask)
        for (int c0 = 0; c0 < a.N; c0 += 64)
            asm volatile("prefetch.global.L2 [%0];" ::"l"(a.mask + orow * a.N + c0));
    if (a.addend)
        for (int c0 = 0; c0 < a.N; c0 += 64)
            asm volatile("prefetch.global.L2 [%0];" ::"l"(a.addend + orow * a.add_stride +
                                                          a.add_off + c0));
}

// ---- the kernel ------------------------------------------------------------
// The weight adjoint is held to 128 registers per thread so that 4 CTAs fit
// per SM (it used 150 unbounded, 3 CTAs; 847 against 915 µs per training
// step, no spills); the other passes are limited by shared memory.
template <int MODE>
__global__ void __launch_bounds__(kThreads, MODE == WGRAD ? 4 : 1) k_conv(const ConvArgs a)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t *sm = reinterpret_cast<uint8_t *>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *sA = sm;
    const int btile = a.N * 128;  // bytes of one B slot: N rows x 64 K
    uint8_t *sB = sA + kStages * kATile;
    uint64_t *bars = reinterpret_cast<uint64_t *>(sB + kStages * btile);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + 2 * kStages + 1);
    int *s_unit0 = reinterpret_cast<int *>(tslot + 1);
    int *s_nst = s_unit0 + kMaxClasses + 1;
    int *s_slice0 = s_nst + kMaxClasses;
    Tables &T = *reinterpret_cast<Tables *>(s_slice0 + kMaxClasses);
    const uint32_t bar_full = smem_u32(bars), bar_free = bar_full + 8 * kStages,
                   bar_done = bar_full + 16 * kStages;
    const int tid = threadIdx.x, warp = tid >> 5;

    if (tid < kMaxClasses + 1)
        s_unit0[tid] = a.cls_unit0[tid < a.classes ? tid : a.classes];
    if (tid < kMaxClasses) {
        s_nst[tid] = a.cls_nst[tid < a.classes ? tid : 0];
        s_slice0[tid] = a.cls_slice0[tid < a.classes ? tid : 0];
    }
    build_tables(a, T, tid, MODE);
    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(bar_full + 8 * s, 1);
            mbar_init(bar_free + 8 * s, 1);
        }
        mbar_init(bar_done, 1);
        fence_mbar_init();
    }
    if (warp == 0) {
        tmem_alloc(smem_u32(tslot), a.tmem_cols);
        tmem_relinquish();
    }
    if (MODE == WGRAD && a.mtiles == 1) {
        // the A rows past the bias row never change: zero them in every slot
        for (int i = tid; i < kStages * kATile / 16; i += kThreads)
            reinterpret_cast<uint4 *>(sA)[i] = make_uint4(0, 0, 0, 0);
    }
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    const uint32_t tmem = *tslot;

    Cursor prod;
    prod.u = blockIdx.x;
    prod.kk = 0;
    cursor_set(prod, a.units, a.classes, s_unit0, s_nst);
    Cursor cons = prod;
    uint32_t pit = 0, cit = 0, nunit = 0;

    UnitState ust;
    if (prod.u < a.units)
        unit_begin<MODE>(a, prod, tid, ust);

    auto produce = [&]() {
        if (prod.u < a.units) {
            const int s = (int)(pit % kStages);
            const uint32_t use = pit / kStages;
            if (use > 0)
                mbar_wait(bar_free + 8 * s, (use - 1) & 1);
            uint8_t *B = sB + s * btile;
            if (MODE != WGRAD && tid == 0) {
                mbar_expect_tx(bar_full + 8 * s, (uint32_t)btile);
                bulk_load(smem_u32(B),
                          a.wpk + (size_t)(s_slice0[prod.cls] + prod.kk) * a.N * kBK,
                          (uint32_t)btile, bar_full + 8 * s);
            }
            fill_item<MODE>(a, prod, ust, sA + s * kATile, B, tid, T.tapoff, T.ctoff,
                            MODE == FWD ? s_slice0[prod.cls] : 0);
            ++pit;
            if (++prod.kk >= prod.nst) {
                prod.kk = 0;
                prod.u += gridDim.x;
                cursor_set(prod, a.units, a.classes, s_unit0, s_nst);
                if (prod.u < a.units)
                    unit_begin<MODE>(a, prod, tid, ust);
            }
        }
        cp_commit();
    };

    // the item gathered at step i goes into the slot whose MMA was issued
    // kStages - kAhead steps earlier, so that wait seldom stalls
#pragma unroll 1
    for (int j = 0; j < kAhead; ++j)
        produce();

#pragma unroll 1
    while (cons.u < a.units) {
        produce();
        cp_wait<kAhead>();
        fence_proxy_async();
        __syncthreads();
        const int s = (int)(cit % kStages);
        const uint32_t use = cit / kStages;
        if (tid == 0) {
            if (MODE != WGRAD)
                mbar_wait(bar_full + 8 * s, use & 1);
            tc_after_sync();
            const uint32_t a0 = smem_u32(sA + s * kATile), b0 = smem_u32(sB + s * btile);
#pragma unroll
            for (int j = 0; j < kBK / 16; ++j)
                tc_mma(tmem, sdesc(a0 + 256 * j), sdesc(b0 + 256 * j), a.idesc,
                       (cons.kk | j) != 0);
            tc_commit(bar_free + 8 * s);
        }
        ++cit;
        if (cons.kk == cons.nst - 1) {
            if (MODE == DGRAD)
                dgrad_prefetch(a, cons, tid);
            if (tid == 0)
                tc_commit(bar_done);
            mbar_wait(bar_done, nunit & 1);
            tc_after_sync();
            epilogue<MODE>(a, cons, tmem + ((uint32_t)(warp * 32) << 16), tid);
            tc_before_sync();
            __syncthreads();
            ++nunit;
        }
        if (++cons.kk >= cons.nst) {
            cons.kk = 0;
            cons.u += gridDim.x;
            cursor_set(cons, a.units, a.classes, s_unit0, s_nst);
        }
    }
    cp_wait<0>();
    __syncthreads();
    if (warp == 0)
        tmem_dealloc(tmem, a.tmem_cols);
}

// Weight slices in the shared-memory layout of the B operand: slice s holds
// rows n < N and K elements [64 s, 64 s + 64), K-major, zero beyond the real
// rows and K. mode 0 (forward): B[n = co][k = t cin + ci] = w[co][t][ci], the
// master layout's own order. mode 1 (dgrad, stride 1): B[n = ci][k = t cout
// + co] = w[co][t][ci]. mode 2 (dgrad, stride 2): the slices of the 8 parity
// classes one after the other, class c over its own taps in the order of
// class_tap.
__device__ __forceinline__ int class_ntaps(int cls)
{
    return (1 + ((cls >> 2) & 1)) * (1 + ((cls >> 1) & 1)) * (1 + (cls & 1));
}

// Tap t (0..26) of tap index ti of a parity class: per odd axis i = 0 is
// d = -1 and i = 1 is d = +1; an even axis has d = 0 only.
__device__ __forceinline__ int class_tap(int cls, int ti)
{
    const int cz = (cls >> 2) & 1, cy = (cls >> 1) & 1, cx = cls & 1;
    const int ny = 1 + cy, nx = 1 + cx;
    const int ix = ti % nx, iy = (ti / nx) % ny, iz = ti / (nx * ny);
    const int dz = cz ? 2 * iz - 1 : 0, dy = cy ? 2 * iy - 1 : 0, dx = cx ? 2 * ix - 1 : 0;
    return (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1);
}

__global__ void k_pack_weights(const float *__restrict__ w, int cin, int cout, int N, int nslices,
                               int mode, __nv_bfloat16 *__restrict__ out)
{
    const int total = nslices * N * kBK;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
        int s = e / (N * kBK);
        const int rem = e - s * N * kBK;
        const int g = rem / 512, r2 = rem - g * 512;
        const int kc = r2 / 64, r3 = r2 - kc * 64;
        const int n = g * 8 + r3 / 8;
        float val = 0.0f;
        if (mode == 0) {
            const int k = s * kBK + kc * 8 + (r3 & 7);
            if (n < cout && k < 27 * cin)
                val = w[(size_t)n * 27 * cin + k];
        } else if (mode == 1) {
            const int k = s * kBK + kc * 8 + (r3 & 7);
            if (n < cin && k < 27 * cout) {
                const int t = k / cout, co = k - t * cout;
                val = w[((size_t)co * 27 + t) * cin + n];
            }
        } else {
            int cls = 0;
            while (cls < 7) {
                const int ns = (class_ntaps(cls) * cout + kBK - 1) / kBK;
                if (s < ns)
                    break;
                s -= ns;
                ++cls;
            }
            const int k = s * kBK + kc * 8 + (r3 & 7);
            if (n < cin && k < class_ntaps(cls) * cout) {
                const int ti = k / cout, co = k - ti * cout;
                val = w[((size_t)co * 27 + class_tap(cls, ti)) * cin + n];
            }
        }
        out[e] = __float2bfloat16_rn(val);
    }
}

// Position of B[n][k] in a packed copy whose slices start at slice s0 and
// hold N rows: slice s0 + k / 64, group of 8 rows n / 8, chunk of 8 K
// elements (k % 64) / 8, row n % 8, element k % 8 (k_pack_weights' layout).
__device__ __forceinline__ int64_t packed_pos(int n, int k, int N, int s0)
{
    const int s = s0 + k / kBK, kk = k % kBK;
    return ((int64_t)s * N + (n / 8) * 8) * kBK + (kk / 8) * 64 + (n % 8) * 8 + (kk & 7);
}

// Adam on a network's flat parameters with k_adam_flat's update, writing each
// updated weight of the listed layers, rounded to bf16, to where
// k_pack_weights puts it: forward B[co][t cin + ci]; dgrad at stride 1
// B[ci][t cout + co]; at stride 2 B[ci][ti cout + co] in the slices of the
// tap's parity class (odd offsets on the axes of the class; ti the tap's index
// within it, x fastest). Each weight has one place per copy, so only real
// weights are written and the zero padding of the previous pack stays.
__global__ void k_adam_pack(AdamPackArgs a, const int64_t *__restrict__ step,
                            float *__restrict__ p, const float *__restrict__ g,
                            float *__restrict__ m, float *__restrict__ v)
{
    __shared__ float s_ib[2];
    if (threadIdx.x == 0) {
        const long long t = (long long)*step + 1;
        s_ib[0] = adam_inv_bias(a.adam.beta1, t);
        s_ib[1] = adam_inv_bias(a.adam.beta2, t);
    }
    __syncthreads();
    const float b1 = (float)a.adam.beta1, b2 = (float)a.adam.beta2;
    const float o1 = (float)(1.0 - a.adam.beta1), o2 = (float)(1.0 - a.adam.beta2);
    const float ib1 = s_ib[0], ib2 = s_ib[1];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.adam.n;
         i += (int64_t)gridDim.x * blockDim.x) {
        float mm = m[i], vv = v[i];
        const float pn =
            adam_flat_update(p[i], g[i], mm, vv, b1, o1, b2, o2, a.adam.lr, a.adam.eps, ib1, ib2);
        p[i] = pn;
        m[i] = mm;
        v[i] = vv;
        for (int j = 0; j < a.nl; ++j) {
            const PackLayer &L = a.L[j];
            const int64_t r = i - L.off;
            const int K = 27 * L.cin;
            if (r < 0 || r >= (int64_t)L.cout * K)
                continue;
            const int co = (int)(r / K), k = (int)(r - (int64_t)co * K);
            const int t = k / L.cin, ci = k - t * L.cin;
            const __nv_bfloat16 b = __float2bfloat16_rn(pn);
            if (L.fwd)
                static_cast<__nv_bfloat16 *>(L.fwd)[packed_pos(co, k, L.cout, 0)] = b;
            if (L.dmode == 1) {
                static_cast<__nv_bfloat16 *>(L.dgrad)[packed_pos(ci, t * L.cout + co, L.cin, 0)] =
                    b;
            } else if (L.dmode == 2) {
                const int tz = t / 9, ty = (t / 3) % 3, tx = t % 3;
                const int cz = tz != 1, cy = ty != 1, cx = tx != 1;
                const int cls = (cz << 2) | (cy << 1) | cx;
                const int ti = ((cz ? tz / 2 : 0) * (1 + cy) + (cy ? ty / 2 : 0)) * (1 + cx) +
                               (cx ? tx / 2 : 0);
                static_cast<__nv_bfloat16 *>(L.dgrad)[packed_pos(ci, ti * L.cout + co, L.cin,
                                                                 L.cls0[cls])] = b;
            }
            break;
        }
    }
}

// g_w[co][t][ci] and g_b[co] from the wgrad partials [split][mrows][N]: one
// block of kReduceThreads per M row m = t cin + ci (m = 27 cin is the bias
// row). Thread j adds the splits j / N, j / N + G, ... of column co = j % N
// (G = kReduceThreads / N groups, coalesced reads of the N columns of a
// split), in order with compensated fp32 sums; the G group sums are then added in order
// by one thread per column, so the result does not depend on timing.
constexpr int kReduceThreads = 512;

// Compensated (Kahan) fp32 accumulation: the sum keeps about the precision of
// one rounding whatever the number of terms, with full-rate fp32 adds (FP64
// issues slowly on this part).
struct Kahan {
    float s = 0.0f, c = 0.0f;
    __device__ __forceinline__ void add(float x)
    {
        const float y = x - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
};

__global__ void __launch_bounds__(kReduceThreads)
    k_wgrad_reduce(const float *__restrict__ part, int splits, int mrows, int N, int cin,
                   int cout, float *__restrict__ gw, float *__restrict__ gb)
{
    __shared__ float red[kReduceThreads];
    const int m = blockIdx.x;
    const int groups = kReduceThreads / N;
    const int co = threadIdx.x % N, grp = threadIdx.x / N;
    Kahan acc;
    if (grp < groups) {
        const float *p = part + (size_t)m * N + co;
        const size_t step = (size_t)mrows * N;
        int sp = grp;
        // four independent loads in flight per thread, added in split order
        for (; sp + 3 * groups < splits; sp += 4 * groups) {
            const float a = p[(size_t)sp * step], b = p[(size_t)(sp + groups) * step],
                        c = p[(size_t)(sp + 2 * groups) * step],
                        d = p[(size_t)(sp + 3 * groups) * step];
            acc.add(a);
            acc.add(b);
            acc.add(c);
            acc.add(d);
        }
        for (; sp < splits; sp += groups)
            acc.add(p[(size_t)sp * step]);
    }
    red[threadIdx.x] = acc.s - acc.c;
    __syncthreads();
    if (threadIdx.x < N && co < cout) {
        Kahan tot;
        for (int gi = 0; gi < groups; ++gi)
            tot.add(red[gi * N + co]);
        const float v = tot.s - tot.c;
        if (m < 27 * cin)
            gw[(size_t)co * 27 * cin + m] = v;
        else if (gb)
            gb[co] = v;
    }
}

// Split-K forward: out[row][n] = act(sum_p part[p][row][n] + bias[n]), the
// partitions added in order; bf16 or fp32 output.
__global__ void k_fwd_reduce(const float *__restrict__ part, int parts, int64_t rows, int N,
                             const float *__restrict__ bias, int relu, int out_f32,
                             void *__restrict__ out)
{
    const int64_t total = rows * N;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        float v = 0.0f;
        for (int p = 0; p < parts; ++p)
            v += part[(size_t)p * total + e];
        if (bias)
            v += __ldg(bias + (int)(e % N));
        if (relu)
            v = fmaxf(v, 0.0f);
        if (out_f32)
            static_cast<float *>(out)[e] = v;
        else
            static_cast<__nv_bfloat16 *>(out)[e] = __float2bfloat16_rn(v);
    }
}

uint32_t make_idesc(int N, bool mn_major)
{
    // kind::f16 instruction descriptor: D fp32 (bits 4-5 = 1), A and B bf16
    // (bits 7-9 = 1, 10-12 = 1), A/B major (bits 15, 16), N >> 3 (bits 17-22),
    // M >> 4 (bits 24-28), M = 128.
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)mn_major << 15) |
           ((uint32_t)mn_major << 16) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

uint32_t tmem_cols_for(int N)
{
    uint32_t c = 32;
    while ((int)c < N)
        c <<= 1;
    return c;
}

// Dynamic shared memory: 1024-byte alignment slack, the ring's A and B
// slots, 2 kStages + 1 mbarriers, the TMEM address, the class tables and
// the tap offset tables.
size_t conv_smem_bytes(int N)
{
    return 1024 + kStages * (size_t)kATile + kStages * (size_t)N * 128 + 8 * (2 * kStages + 1) +
           4 + 4 * (3 * kMaxClasses + 1) + sizeof(Tables);
}

// Parity classes of the stride-2 dgrad (host side): units, K slices and
// first packed slice of each class; returns the total number of units.
int dgrad_classes(const ConvLayer &l, int *unit0, int *nst, int *slice0, int *total_slices)
{
    int u = 0, sl = 0;
    for (int c = 0; c < kMaxClasses; ++c) {
        const int cz = (c >> 2) & 1, cy = (c >> 1) & 1, cx = c & 1;
        const int64_t rows = (int64_t)l.nb * ((l.D - cz + 1) / 2) * ((l.H - cy + 1) / 2) *
                             ((l.W - cx + 1) / 2);
        const int ntaps = (1 + cz) * (1 + cy) * (1 + cx);
        unit0[c] = u;
        nst[c] = (ntaps * l.cout + kBK - 1) / kBK;
        slice0[c] = sl;
        u += (int)((rows + 127) / 128);
        sl += nst[c];
    }
    unit0[kMaxClasses] = u;
    if (total_slices)
        *total_slices = sl;
    return u;
}

struct DevInfo {
    int sms = 0;
    int occ[3][kMaxN / 16 + 1] = {};
};
std::mutex g_info_mu;
DevInfo g_info[64];

template <int MODE>
cudaError_t grid_for(int N, int units, int *grid)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return e;
    if (dev < 0 || dev >= 64)
        return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_info_mu);
    DevInfo &d = g_info[dev];
    if (d.sms == 0) {
        e = cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess)
            return e;
    }
    int &occ = d.occ[MODE][N / 16];
    if (occ == 0) {
        // resident CTAs per SM from the kernel's own limits: shared memory
        // (with the largest carveout), registers, and TMEM columns (512 per SM)
        e = cudaFuncSetAttribute(k_conv<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)conv_smem_bytes(kMaxN));
        if (e != cudaSuccess)
            return e;
        e = cudaFuncSetAttribute(k_conv<MODE>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
        if (e != cudaSuccess)
            return e;
        cudaFuncAttributes fa;
        e = cudaFuncGetAttributes(&fa, k_conv<MODE>);
        if (e != cudaSuccess)
            return e;
        int smem_sm = 0, resv = 0;
        e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        if (e != cudaSuccess)
            return e;
        e = cudaDeviceGetAttribute(&resv, cudaDevAttrReservedSharedMemoryPerBlock, dev);
        if (e != cudaSuccess)
            return e;
        const int by_smem = smem_sm / (int)(conv_smem_bytes(N) + fa.sharedSizeBytes + resv);
        const int regs_warp = (fa.numRegs * 32 + 255) / 256 * 256;
        const int by_regs = 65536 / (regs_warp * (kThreads / 32));
        const int by_tmem = 512 / (int)tmem_cols_for(N);
        occ = by_smem < by_regs ? by_smem : by_regs;
        occ = occ < by_tmem ? occ : by_tmem;
        occ = occ < 16 ? occ : 16;
        if (occ < 1)
            return cudaErrorInvalidConfiguration;
    }
    *grid = units < d.sms * occ ? units : d.sms * occ;
    return cudaSuccess;
}

int blocks_for(int64_t n, int threads)
{
    int64_t b = (n + threads - 1) / threads;
    if (b > 32 * (int64_t)device_sms())  // grid-stride loops beyond this
        b = 32 * (int64_t)device_sms();
    return (int)(b < 1 ? 1 : b);
}

}  // namespace

int conv_out_size(int n, int stride) { return (n - 1) / stride + 1; }

int conv_slices(int kreal) { return (kreal + kBK - 1) / kBK; }

size_t conv_packed_elems(const ConvLayer &l, int dgrad)
{
    if (!dgrad)
        return (size_t)conv_slices(27 * l.cin) * l.cout * kBK;
    if (l.stride == 1)
        return (size_t)conv_slices(27 * l.cout) * l.cin * kBK;
    int u0[kMaxClasses + 1], ns[kMaxClasses], s0[kMaxClasses], total = 0;
    dgrad_classes(l, u0, ns, s0, &total);
    return (size_t)total * l.cin * kBK;
}

void conv_wgrad_plan(const ConvLayer &l, int *mtiles, int *splits, int *kper)
{
    const int64_t V = (int64_t)l.nb * conv_out_size(l.D, l.stride) * conv_out_size(l.H, l.stride) *
                      conv_out_size(l.W, l.stride);
    const int mt = (27 * l.cin + 1 + 127) / 128;
    int64_t sp = (kTargetUnits + mt - 1) / mt;
    const int64_t max_sp = (V + kBK - 1) / kBK;
    if (sp > max_sp)
        sp = max_sp;
    if (sp < 1)
        sp = 1;
    int64_t kp = (V + sp - 1) / sp;
    kp = (kp + kBK - 1) / kBK * kBK;
    *mtiles = mt;
    *kper = (int)kp;
    *splits = (int)((V + kp - 1) / kp);
}

size_t conv_wgrad_ws_bytes(const ConvLayer &l)
{
    int mt, sp, kp;
    conv_wgrad_plan(l, &mt, &sp, &kp);
    return (size_t)sp * mt * 128 * l.cout * sizeof(float);
}

cudaError_t launch_conv_pack(const ConvLayer &l, const float *w, void *fwd, void *dgrad,
                             cudaStream_t s)
{
    ProfScope ps(s, "k_pack_weights");
    if (fwd) {
        const int nst = conv_slices(27 * l.cin);
        k_pack_weights<<<blocks_for((int64_t)nst * l.cout * kBK, 256), 256, 0, s>>>(
            w, l.cin, l.cout, l.cout, nst, 0, static_cast<__nv_bfloat16 *>(fwd));
    }
    if (dgrad) {
        const int nst = (int)(conv_packed_elems(l, 1) / ((size_t)l.cin * kBK));
        k_pack_weights<<<blocks_for((int64_t)nst * l.cin * kBK, 256), 256, 0, s>>>(
            w, l.cin, l.cout, l.cin, nst, l.stride == 1 ? 1 : 2,
            static_cast<__nv_bfloat16 *>(dgrad));
    }
    return cudaGetLastError();
}

void adam_pack_layer(const ConvLayer &l, int64_t off, void *fwd, void *dgrad, PackLayer *L)
{
    *L = PackLayer{};
    L->off = off;
    L->cin = l.cin;
    L->cout = l.cout;
    L->fwd = fwd;
    L->dgrad = dgrad;
    L->dmode = dgrad ? (l.stride == 1 ? 1 : 2) : 0;
    if (L->dmode == 2) {
        int u0[kMaxClasses + 1], ns[kMaxClasses];
        dgrad_classes(l, u0, ns, L->cls0, nullptr);
    }
}

cudaError_t launch_adam_pack(const AdamPackArgs &a, int64_t *step, float *p, const float *g,
                             float *m, float *v, cudaStream_t s)
{
    {
        ProfScope ps(s, "k_adam_pack");
        k_adam_pack<<<blocks_for(a.adam.n, 256), 256, 0, s>>>(a, step, p, g, m, v);
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return e;
    return launch_step_tick(step, s);
}

static ConvArgs base_args(const ConvLayer &l)
{
    ConvArgs a = {};
    a.D = l.D;
    a.H = l.H;
    a.W = l.W;
    a.Do = conv_out_size(l.D, l.stride);
    a.Ho = conv_out_size(l.H, l.stride);
    a.Wo = conv_out_size(l.W, l.stride);
    a.cin = l.cin;
    a.cout = l.cout;
    a.stride = l.stride;
    a.classes = 1;
    return a;
}

// One class covering every unit, nst slices each.
static void single_class(ConvArgs &a, int nst)
{
    a.classes = 1;
    a.cls_unit0[0] = 0;
    a.cls_unit0[1] = a.units;
    a.cls_nst[0] = nst;
    a.cls_slice0[0] = 0;
}

// K partitions of the forward pass: split only when the tiles alone give
// fewer than two per SM of a 152-SM GB300, at least two K slices per
// partition, at most 8; a function of the shape only, so workspace sizes and
// launches agree.
int conv_fwd_splits(const ConvLayer &l)
{
    const int64_t rows = (int64_t)l.nb * conv_out_size(l.D, l.stride) *
                         conv_out_size(l.H, l.stride) * conv_out_size(l.W, l.stride);
    const int64_t tiles = (rows + 127) / 128;
    const int nst = conv_slices(27 * l.cin);
    if (tiles >= 2 * 152 || nst < 4)
        return 1;
    int64_t sp = (kTargetUnits + tiles - 1) / tiles;
    if (sp > nst / 2)
        sp = nst / 2;
    if (sp > kMaxClasses)
        sp = kMaxClasses;
    return sp < 2 ? 1 : (int)sp;
}

size_t conv_fwd_ws_bytes(const ConvLayer &l)
{
    const int sp = conv_fwd_splits(l);
    if (sp == 1)
        return 0;
    const int64_t rows = (int64_t)l.nb * conv_out_size(l.D, l.stride) *
                         conv_out_size(l.H, l.stride) * conv_out_size(l.W, l.stride);
    return (size_t)sp * rows * l.cout * sizeof(float);
}

cudaError_t launch_conv_forward(const ConvLayer &l, const void *in, const void *wpk,
                                const float *bias, int relu, int out_f32, void *out, void *ws,
                                cudaStream_t s)
{
    ConvArgs a = base_args(l);
    a.act_elems = (int64_t)l.nb * l.D * l.H * l.W * l.cin;
    a.act = static_cast<const __nv_bfloat16 *>(in);
    a.wpk = static_cast<const __nv_bfloat16 *>(wpk);
    a.bias = bias;
    a.out = out;
    a.N = l.cout;
    a.Kreal = 27 * l.cin;
    a.rows = l.nb * a.Do * a.Ho * a.Wo;
    const int tiles = (a.rows + 127) / 128;
    const int nst = conv_slices(a.Kreal);
    const int sp = ws ? conv_fwd_splits(l) : 1;
    if (sp == 1) {
        a.units = tiles;
        single_class(a, nst);
    } else {
        // K partitions as classes over the same tiles: partition p has the
        // slices [p nst / sp, (p + 1) nst / sp)
        a.part = static_cast<float *>(ws);
        a.classes = sp;
        for (int p = 0; p < sp; ++p) {
            a.cls_unit0[p] = p * tiles;
            a.cls_slice0[p] = p * nst / sp;
            a.cls_nst[p] = (p + 1) * nst / sp - p * nst / sp;
        }
        a.cls_unit0[sp] = sp * tiles;
        a.units = sp * tiles;
    }
    a.relu = relu;
    a.out_f32 = out_f32;
    a.idesc = make_idesc(a.N, false);
    a.tmem_cols = tmem_cols_for(a.N);
    int grid = 0;
    cudaError_t e = grid_for<FWD>(a.N, a.units, &grid);
    if (e != cudaSuccess)
        return e;
    {
        ProfScope ps(s, "k_conv_fwd");
        k_conv<FWD><<<grid, kThreads, conv_smem_bytes(a.N), s>>>(a);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess || sp == 1)
        return e;
    ProfScope ps(s, "k_fwd_reduce");
    k_fwd_reduce<<<blocks_for((int64_t)a.rows * a.N, 256), 256, 0, s>>>(
        a.part, sp, a.rows, a.N, bias, relu, out_f32, out);
    return cudaGetLastError();
}

cudaError_t launch_conv_dgrad(const ConvLayer &l, const void *gout, const void *wpk,
                              const void *mask, const void *addend, int add_stride, int add_off,
                              void *gin, cudaStream_t s)
{
    ConvArgs a = base_args(l);
    a.act_elems = (int64_t)l.nb * a.Do * a.Ho * a.Wo * l.cout;
    a.act = static_cast<const __nv_bfloat16 *>(gout);
    a.wpk = static_cast<const __nv_bfloat16 *>(wpk);
    a.mask = static_cast<const __nv_bfloat16 *>(mask);
    a.addend = static_cast<const __nv_bfloat16 *>(addend);
    a.add_stride = add_stride;
    a.add_off = add_off;
    a.out = gin;
    a.N = l.cin;
    a.Kreal = 27 * l.cout;
    a.rows = l.nb * l.D * l.H * l.W;
    if (l.stride == 1) {
        a.units = (a.rows + 127) / 128;
        single_class(a, conv_slices(a.Kreal));
    } else {
        a.classes = kMaxClasses;
        a.units = dgrad_classes(l, a.cls_unit0, a.cls_nst, a.cls_slice0, nullptr);
    }
    a.idesc = make_idesc(a.N, false);
    a.tmem_cols = tmem_cols_for(a.N);
    int grid = 0;
    cudaError_t e = grid_for<DGRAD>(a.N, a.units, &grid);
    if (e != cudaSuccess)
        return e;
    ProfScope ps(s, "k_conv_dgrad");
    k_conv<DGRAD><<<grid, kThreads, conv_smem_bytes(a.N), s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_conv_wgrad(const ConvLayer &l, const void *in, const void *gout, float *gw,
                              float *gb, void *ws, cudaStream_t s)
{
    ConvArgs a = base_args(l);
    a.act_elems = (int64_t)l.nb * l.D * l.H * l.W * l.cin;
    a.gout_elems = (int64_t)l.nb * a.Do * a.Ho * a.Wo * l.cout;
    int mt, sp, kp;
    conv_wgrad_plan(l, &mt, &sp, &kp);
    a.act = static_cast<const __nv_bfloat16 *>(in);
    a.gout = static_cast<const __nv_bfloat16 *>(gout);
    a.out = ws;
    a.N = l.cout;
    a.Kreal = kp;
    a.rows = l.nb * a.Do * a.Ho * a.Wo;
    a.mtiles = mt;
    a.units = mt * sp;
    single_class(a, kp / kBK);
    a.idesc = make_idesc(a.N, true);
    a.tmem_cols = tmem_cols_for(a.N);
    int grid = 0;
    cudaError_t e = grid_for<WGRAD>(a.N, a.units, &grid);
    if (e != cudaSuccess)
        return e;
    {
        ProfScope ps(s, "k_conv_wgrad");
        k_conv<WGRAD><<<grid, kThreads, conv_smem_bytes(a.N), s>>>(a);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess)
        return e;
    ProfScope ps(s, "k_wgrad_reduce");
    // one block per M row (27 cin weights rows and the bias row)
    k_wgrad_reduce<<<27 * l.cin + 1, kReduceThreads, 0, s>>>(static_cast<const float *>(ws), sp,
                                                             mt * 128, a.N, l.cin, l.cout, gw, gb);
    return cudaGetLastError();
}

int conv_device_error(bool clear)
{
    int h = 0;
    if (cudaMemcpyFromSymbol(&h, g_conv_error, sizeof(int)) != cudaSuccess)
        return -1;
    if (h != 0 && clear) {
        const int zero = 0;
        if (cudaMemcpyToSymbol(g_conv_error, &zero, sizeof(int)) != cudaSuccess)
            return -1;
    }
    return h;
}

AL_UNIT_ERROR_READER(unit_error_conv)

}  // namespace airgb
