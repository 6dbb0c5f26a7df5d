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
//             M = input voxels,  N = cin,  K = 27 cout (k = t cout + co)
//             (terms whose (p - d_t)/s is not an integer in range are 0)
//   wgrad     g_w[(t,ci)][co] = sum_o in[s o + d_t][ci] * g_out[o][co]
//             M = 27 cin (+1: a row of ones gives the bias gradient),
//             N = cout, K = output voxels (split over blocks, partials
//             summed in a fixed order by k_wgrad_reduce)
//
// Activations are bf16, channels last ([b][z][y][x][c]); accumulation is
// fp32 in tensor memory. One CTA of 4 warps owns a 128-row tile of D in TMEM
// (tcgen05.alloc), stages K in slices of 64 through a 3-deep shared-memory
// ring, and one thread issues tcgen05.mma (kind::f16, bf16 x bf16 -> f32,
// M = 128, K = 16 per instruction) on shared-memory descriptors; a
// tcgen05.commit per slice frees its ring slot, and the epilogue reads D
// back with tcgen05.ld. The weight operand of the forward and dgrad passes
// is stored pre-tiled in the shared-memory layout, so each slice of it
// arrives with one cp.async.bulk on an mbarrier; the im2col operand is
// gathered by the threads (16-byte loads, zero padding at the faces).
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
constexpr int kStages = 3;
constexpr int kBK = 64;                       // K elements per ring slot
constexpr int kATile = 128 * kBK * 2;         // bytes of one A slot (16 KB)
constexpr int kTargetUnits = 1216;            // wgrad blocks aimed at: 152 SMs x 8
constexpr int kMaxN = 128;
constexpr int kErrTimeout = 6;                // AL_ERR_TIMEOUT

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
    int Kreal;                   // FWD 27 cin, DGRAD 27 cout, WGRAD voxels per split
    int nst;                     // ring slots (K slices of 64) per unit
    int units, mtiles;           // work units; WGRAD: M tiles (units = mtiles x splits)
    int rows;                    // FWD: output voxels; DGRAD: input voxels; WGRAD: output voxels
    int relu, out_f32, add_stride, add_off;
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

__device__ __forceinline__ uint4 ldg16(const __nv_bfloat16 *p)
{
    return __ldg(reinterpret_cast<const uint4 *>(p));
}

__device__ __forceinline__ void sts16(uint8_t *p, const uint4 &v)
{
    *reinterpret_cast<uint4 *>(p) = v;
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

// ---- operand fills ---------------------------------------------------------
// One 16-byte group of 8 consecutive channels [c0, c0 + 8) of voxel (b, z, y,
// x) of a channels-last volume with C channels, zero outside the grid.
__device__ __forceinline__ uint4 load_group(const __nv_bfloat16 *__restrict__ v, int b, int z,
                                            int y, int x, int D, int H, int W, int C, int c0)
{
    if (z < 0 || z >= D || y < 0 || y >= H || x < 0 || x >= W)
        return make_uint4(0, 0, 0, 0);
    return ldg16(v + ((((size_t)b * D + z) * H + y) * W + x) * C + c0);
}

// Same for C not a multiple of 8: element e of the group is flat index
// first + e of the (tap, channel) sequence, each an individual 2-byte load.
// Used by the 2-channel input layer only.
__device__ __forceinline__ uint4 load_group_scalar(const __nv_bfloat16 *__restrict__ v, int b,
                                                   int z0, int y0, int x0, int D, int H, int W,
                                                   int C, int first, int kend)
{
    uint32_t w[4] = {0, 0, 0, 0};
    const uint16_t *raw = reinterpret_cast<const uint16_t *>(v);
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        const int k = first + e;
        if (k >= kend)
            break;
        const int t = k / C, c = k - t * C;
        const int z = z0 + t / 9, y = y0 + (t / 3) % 3, x = x0 + t % 3;
        if (z < 0 || z >= D || y < 0 || y >= H || x < 0 || x >= W)
            continue;
        const uint32_t h = __ldg(raw + ((((size_t)b * D + z) * H + y) * W + x) * C + c);
        w[e >> 1] |= h << (16 * (e & 1));
    }
    return make_uint4(w[0], w[1], w[2], w[3]);
}

// ---- the kernel ------------------------------------------------------------
template <int MODE>
__global__ void __launch_bounds__(kThreads) k_conv(const ConvArgs a)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t *sm = reinterpret_cast<uint8_t *>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *sA = sm;
    const int btile = a.N * 128;  // bytes of one B slot: N rows x 64 K
    uint8_t *sB = sA + kStages * kATile;
    uint64_t *bars = reinterpret_cast<uint64_t *>(sB + kStages * btile);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + 2 * kStages + 1);
    const uint32_t bar_full = smem_u32(bars), bar_free = bar_full + 8 * kStages,
                   bar_done = bar_full + 16 * kStages;
    const int tid = threadIdx.x, warp = tid >> 5;

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
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    const uint32_t tmem = *tslot;

    uint32_t it = 0, nunit = 0;
    for (int u = blockIdx.x; u < a.units; u += gridDim.x, ++nunit) {
        // ---- per-unit geometry ----
        int row = 0, b = 0, z0 = 0, y0 = 0, x0 = 0;
        bool valid = false;
        int mt = 0, vbeg = 0, vend = 0;
        if (MODE == FWD || MODE == DGRAD) {
            row = u * 128 + tid;
            valid = row < a.rows;
            int r = valid ? row : 0;
            const int X = MODE == FWD ? a.Wo : a.W, Y = MODE == FWD ? a.Ho : a.H,
                      Z = MODE == FWD ? a.Do : a.D;
            const int x = r % X;
            r /= X;
            const int y = r % Y;
            r /= Y;
            const int z = r % Z;
            b = r / Z;
            if (MODE == FWD) {
                z0 = z * a.stride - 1;
                y0 = y * a.stride - 1;
                x0 = x * a.stride - 1;
            } else {
                z0 = z;
                y0 = y;
                x0 = x;
            }
        } else {
            mt = u % a.mtiles;
            vbeg = (u / a.mtiles) * a.Kreal;
            vend = min(vbeg + a.Kreal, a.rows);
        }

        for (int kk = 0; kk < a.nst; ++kk, ++it) {
            const int s = (int)(it % kStages);
            const uint32_t use = it / kStages;
            if (use > 0)
                mbar_wait(bar_free + 8 * s, (use - 1) & 1);
            uint8_t *A = sA + s * kATile;
            uint8_t *B = sB + s * btile;
            if (MODE != WGRAD && tid == 0) {
                mbar_expect_tx(bar_full + 8 * s, (uint32_t)btile);
                bulk_load(smem_u32(B), a.wpk + (size_t)kk * a.N * kBK, (uint32_t)btile,
                          bar_full + 8 * s);
            }
            if (MODE == FWD) {
                uint4 v[8];
                const int k0 = kk * kBK;
                if ((a.cin & 7) == 0) {
#pragma unroll
                    for (int kc = 0; kc < 8; ++kc) {
                        const int k = k0 + kc * 8;
                        v[kc] = make_uint4(0, 0, 0, 0);
                        if (valid && k < a.Kreal) {
                            const int t = k / a.cin, c = k - t * a.cin;
                            v[kc] = load_group(a.act, b, z0 + t / 9, y0 + (t / 3) % 3, x0 + t % 3,
                                               a.D, a.H, a.W, a.cin, c);
                        }
                    }
                } else {
#pragma unroll
                    for (int kc = 0; kc < 8; ++kc)
                        v[kc] = valid ? load_group_scalar(a.act, b, z0, y0, x0, a.D, a.H, a.W,
                                                          a.cin, k0 + kc * 8, a.Kreal)
                                      : make_uint4(0, 0, 0, 0);
                }
#pragma unroll
                for (int kc = 0; kc < 8; ++kc)
                    sts16(A + kmajor_off(tid, kc), v[kc]);
            } else if (MODE == DGRAD) {
                uint4 v[8];
                const int k0 = kk * kBK;
#pragma unroll
                for (int kc = 0; kc < 8; ++kc) {
                    const int k = k0 + kc * 8;
                    v[kc] = make_uint4(0, 0, 0, 0);
                    if (valid && k < a.Kreal) {
                        const int t = k / a.cout, c = k - t * a.cout;
                        // output voxel o with s o + d = p, per axis
                        const int nz = z0 - (t / 9 - 1), ny = y0 - ((t / 3) % 3 - 1),
                                  nx = x0 - (t % 3 - 1);
                        const bool ok = a.stride == 1 ? true
                                                      : (nz >= 0 && ny >= 0 && nx >= 0 &&
                                                         ((nz | ny | nx) & 1) == 0);
                        if (ok)
                            v[kc] = load_group(a.act, b, nz / a.stride, ny / a.stride,
                                               nx / a.stride, a.Do, a.Ho, a.Wo, a.cout, c);
                    }
                }
#pragma unroll
                for (int kc = 0; kc < 8; ++kc)
                    sts16(A + kmajor_off(tid, kc), v[kc]);
            } else {
                // A: rows m = (t, ci) of M tile mt, K = 64 voxels from vbeg + 64 kk.
                // 16 M groups x 64 K rows = 1024 16-byte rows, 8 per thread.
                const int kbase = vbeg + kk * kBK;
                const int kreal = 27 * a.cin;
#pragma unroll 2
                for (int i = 0; i < 8; ++i) {
                    const int idx = tid + i * kThreads;
                    const int krow = idx & 7, cm = idx >> 3;
                    const int g = cm & 15, kg = cm >> 4;
                    const int k = kg * 8 + krow;
                    const int vox = kbase + k;
                    const int m0 = mt * 128 + g * 8;
                    uint4 val = make_uint4(0, 0, 0, 0);
                    if (vox < vend) {
                        int r = vox;
                        const int ox = r % a.Wo;
                        r /= a.Wo;
                        const int oy = r % a.Ho;
                        r /= a.Ho;
                        const int oz = r % a.Do;
                        const int bb = r / a.Do;
                        const int zz = oz * a.stride - 1, yy = oy * a.stride - 1,
                                  xx = ox * a.stride - 1;
                        if ((a.cin & 7) == 0) {
                            if (m0 < kreal) {
                                const int t = m0 / a.cin, c = m0 - t * a.cin;
                                val = load_group(a.act, bb, zz + t / 9, yy + (t / 3) % 3,
                                                 xx + t % 3, a.D, a.H, a.W, a.cin, c);
                            } else if (m0 == kreal) {
                                val.x = 0x3F80u;  // bf16 1.0 in element 0: the bias row
                            }
                        } else {
                            val = load_group_scalar(a.act, bb, zz, yy, xx, a.D, a.H, a.W, a.cin,
                                                    m0, kreal);
                            if (m0 <= kreal && kreal < m0 + 8) {
                                const int e = kreal - m0;
                                const uint32_t one = 0x3F80u << (16 * (e & 1));
                                switch (e >> 1) {
                                case 0: val.x |= one; break;
                                case 1: val.y |= one; break;
                                case 2: val.z |= one; break;
                                default: val.w |= one; break;
                                }
                            }
                        }
                    }
                    sts16(A + mnmajor_off(g, k), val);
                }
                // B: rows n = co (N / 8 groups) x 64 voxels.
                const int ng = a.N >> 3;
                for (int idx = tid; idx < ng * kBK; idx += kThreads) {
                    const int krow = idx & 7, cm = idx >> 3;
                    const int g = cm % ng, kg = cm / ng;
                    const int k = kg * 8 + krow;
                    const int vox = kbase + k;
                    uint4 val = make_uint4(0, 0, 0, 0);
                    if (vox < vend)
                        val = ldg16(a.gout + (size_t)vox * a.cout + g * 8);
                    sts16(B + mnmajor_off(g, k), val);
                }
            }
            fence_proxy_async();
            __syncthreads();
            if (tid == 0) {
                if (MODE != WGRAD)
                    mbar_wait(bar_full + 8 * s, use & 1);
                tc_after_sync();
                const uint32_t a0 = smem_u32(A), b0 = smem_u32(B);
#pragma unroll
                for (int j = 0; j < kBK / 16; ++j)
                    tc_mma(tmem, sdesc(a0 + 256 * j), sdesc(b0 + 256 * j), a.idesc,
                           (kk | j) != 0);
                tc_commit(bar_free + 8 * s);
            }
        }
        if (tid == 0)
            tc_commit(bar_done);
        mbar_wait(bar_done, nunit & 1);
        tc_after_sync();

        // ---- epilogue: row tid of the tile from TMEM lane tid ----
        const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
        for (int c0 = 0; c0 < a.N; c0 += 16) {
            float v[16];
            tc_load16(lane_addr + (uint32_t)c0, v);
            if (MODE == FWD) {
                if (!valid)
                    continue;
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
                if (a.out_f32) {
                    float4 *o = reinterpret_cast<float4 *>(static_cast<float *>(a.out) +
                                                           (size_t)row * a.N + c0);
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        o[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
                } else {
                    uint4 *o = reinterpret_cast<uint4 *>(static_cast<__nv_bfloat16 *>(a.out) +
                                                         (size_t)row * a.N + c0);
                    o[0] = make_uint4(pack_bf16(v[0], v[1]), pack_bf16(v[2], v[3]),
                                      pack_bf16(v[4], v[5]), pack_bf16(v[6], v[7]));
                    o[1] = make_uint4(pack_bf16(v[8], v[9]), pack_bf16(v[10], v[11]),
                                      pack_bf16(v[12], v[13]), pack_bf16(v[14], v[15]));
                }
            } else if (MODE == DGRAD) {
                if (!valid)
                    continue;
                if (a.addend) {
                    const uint4 *p = reinterpret_cast<const uint4 *>(
                        a.addend + (size_t)row * a.add_stride + a.add_off + c0);
#pragma unroll
                    for (int q = 0; q < 2; ++q) {
                        const uint4 w = __ldg(p + q);
                        v[8 * q + 0] += bf16_lo(w.x);
                        v[8 * q + 1] += bf16_hi(w.x);
                        v[8 * q + 2] += bf16_lo(w.y);
                        v[8 * q + 3] += bf16_hi(w.y);
                        v[8 * q + 4] += bf16_lo(w.z);
                        v[8 * q + 5] += bf16_hi(w.z);
                        v[8 * q + 6] += bf16_lo(w.w);
                        v[8 * q + 7] += bf16_hi(w.w);
                    }
                }
                if (a.mask) {
                    const uint4 *p =
                        reinterpret_cast<const uint4 *>(a.mask + (size_t)row * a.N + c0);
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
                uint4 *o = reinterpret_cast<uint4 *>(static_cast<__nv_bfloat16 *>(a.out) +
                                                     (size_t)row * a.N + c0);
                o[0] = make_uint4(pack_bf16(v[0], v[1]), pack_bf16(v[2], v[3]),
                                  pack_bf16(v[4], v[5]), pack_bf16(v[6], v[7]));
                o[1] = make_uint4(pack_bf16(v[8], v[9]), pack_bf16(v[10], v[11]),
                                  pack_bf16(v[12], v[13]), pack_bf16(v[14], v[15]));
            } else {
                const int split = u / a.mtiles;
                const size_t m = (size_t)split * a.mtiles * 128 + (size_t)mt * 128 + tid;
                float4 *o = reinterpret_cast<float4 *>(static_cast<float *>(a.out) + m * a.N + c0);
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    o[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
            }
        }
        tc_before_sync();
        __syncthreads();
    }
    if (warp == 0)
        tmem_dealloc(tmem, a.tmem_cols);
}

// Weight slices in the shared-memory layout of the B operand: slice s holds
// rows n < N and K elements [64 s, 64 s + 64), K-major, zero beyond the real
// rows and K. fwd: B[n = co][k = t cin + ci] = w[co][t][ci] (the master
// layout's own order); dgrad: B[n = ci][k = t cout + co] = w[co][t][ci].
__global__ void k_pack_weights(const float *__restrict__ w, int cin, int cout, int N, int nst,
                               int dgrad, __nv_bfloat16 *__restrict__ out)
{
    const int total = nst * N * kBK;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
        const int s = e / (N * kBK), rem = e - s * N * kBK;
        const int g = rem / 512, r2 = rem - g * 512;
        const int kc = r2 / 64, r3 = r2 - kc * 64;
        const int n = g * 8 + r3 / 8, k = s * kBK + kc * 8 + (r3 & 7);
        float val = 0.0f;
        if (!dgrad) {
            if (n < cout && k < 27 * cin)
                val = w[(size_t)n * 27 * cin + k];
        } else if (n < cin && k < 27 * cout) {
            const int t = k / cout, co = k - t * cout;
            val = w[((size_t)co * 27 + t) * cin + n];
        }
        out[e] = __float2bfloat16_rn(val);
    }
}

// g_w[co][t][ci] and g_b[co] from the wgrad partials [split][mtiles*128][N],
// summed over the splits in order, in double.
__global__ void k_wgrad_reduce(const float *__restrict__ part, int splits, int mrows, int N,
                               int cin, int cout, float *__restrict__ gw, float *__restrict__ gb)
{
    const int nw = cout * 27 * cin;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nw + cout;
         e += gridDim.x * blockDim.x) {
        int m, co;
        if (e < nw) {
            co = e / (27 * cin);
            m = e - co * 27 * cin;  // t cin + ci
        } else {
            co = e - nw;
            m = 27 * cin;
        }
        double acc = 0.0;
        for (int s = 0; s < splits; ++s)
            acc += (double)part[((size_t)s * mrows + m) * N + co];
        if (e < nw)
            gw[e] = (float)acc;
        else if (gb)
            gb[co] = (float)acc;
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

size_t conv_smem_bytes(int N) { return 1024 + kStages * (size_t)kATile + kStages * (size_t)N * 128 + 64; }

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
        e = cudaFuncSetAttribute(k_conv<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)conv_smem_bytes(kMaxN));
        if (e != cudaSuccess)
            return e;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_conv<MODE>, kThreads,
                                                          conv_smem_bytes(N));
        if (e != cudaSuccess)
            return e;
        if (occ < 1)
            return cudaErrorInvalidConfiguration;
    }
    *grid = units < d.sms * occ ? units : d.sms * occ;
    return cudaSuccess;
}

int blocks_for(int64_t n, int threads)
{
    int64_t b = (n + threads - 1) / threads;
    if (b > 152 * 32)
        b = 152 * 32;
    return (int)(b < 1 ? 1 : b);
}

}  // namespace

int conv_out_size(int n, int stride) { return (n - 1) / stride + 1; }

int conv_slices(int kreal) { return (kreal + kBK - 1) / kBK; }

size_t conv_packed_elems(const ConvLayer &l, int dgrad)
{
    const int N = dgrad ? l.cin : l.cout;
    return (size_t)conv_slices(27 * (dgrad ? l.cout : l.cin)) * N * kBK;
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
        const int nst = conv_slices(27 * l.cout);
        k_pack_weights<<<blocks_for((int64_t)nst * l.cin * kBK, 256), 256, 0, s>>>(
            w, l.cin, l.cout, l.cin, nst, 1, static_cast<__nv_bfloat16 *>(dgrad));
    }
    return cudaGetLastError();
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
    return a;
}

cudaError_t launch_conv_forward(const ConvLayer &l, const void *in, const void *wpk,
                                const float *bias, int relu, int out_f32, void *out, cudaStream_t s)
{
    ConvArgs a = base_args(l);
    a.act = static_cast<const __nv_bfloat16 *>(in);
    a.wpk = static_cast<const __nv_bfloat16 *>(wpk);
    a.bias = bias;
    a.out = out;
    a.N = l.cout;
    a.Kreal = 27 * l.cin;
    a.nst = conv_slices(a.Kreal);
    a.rows = l.nb * a.Do * a.Ho * a.Wo;
    a.units = (a.rows + 127) / 128;
    a.relu = relu;
    a.out_f32 = out_f32;
    a.idesc = make_idesc(a.N, false);
    a.tmem_cols = tmem_cols_for(a.N);
    int grid = 0;
    cudaError_t e = grid_for<FWD>(a.N, a.units, &grid);
    if (e != cudaSuccess)
        return e;
    ProfScope ps(s, "k_conv_fwd");
    k_conv<FWD><<<grid, kThreads, conv_smem_bytes(a.N), s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_conv_dgrad(const ConvLayer &l, const void *gout, const void *wpk,
                              const void *mask, const void *addend, int add_stride, int add_off,
                              void *gin, cudaStream_t s)
{
    ConvArgs a = base_args(l);
    a.act = static_cast<const __nv_bfloat16 *>(gout);
    a.wpk = static_cast<const __nv_bfloat16 *>(wpk);
    a.mask = static_cast<const __nv_bfloat16 *>(mask);
    a.addend = static_cast<const __nv_bfloat16 *>(addend);
    a.add_stride = add_stride;
    a.add_off = add_off;
    a.out = gin;
    a.N = l.cin;
    a.Kreal = 27 * l.cout;
    a.nst = conv_slices(a.Kreal);
    a.rows = l.nb * l.D * l.H * l.W;
    a.units = (a.rows + 127) / 128;
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
    int mt, sp, kp;
    conv_wgrad_plan(l, &mt, &sp, &kp);
    a.act = static_cast<const __nv_bfloat16 *>(in);
    a.gout = static_cast<const __nv_bfloat16 *>(gout);
    a.out = ws;
    a.N = l.cout;
    a.Kreal = kp;
    a.nst = kp / kBK;
    a.rows = l.nb * a.Do * a.Ho * a.Wo;
    a.mtiles = mt;
    a.units = mt * sp;
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
    k_wgrad_reduce<<<blocks_for((int64_t)l.cout * 27 * l.cin + l.cout, 256), 256, 0, s>>>(
        static_cast<const float *>(ws), sp, mt * 128, a.N, l.cin, l.cout, gw, gb);
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

}  // namespace airgb
