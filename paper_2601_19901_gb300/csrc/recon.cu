// Learned angular reconstruction: the U-Net's layers on the 5th-generation
// tensor cores (tcgen05: BF16 operands in shared memory, FP32 accumulators in
// tensor memory), operands staged by TMA.
//
// Activation layout. Every activation of resolution level l is a bordered
// image of (Hl + 2) x (Wl + 2) positions q = y (Wl + 2) + x: the level's
// Hl x Wl image with a ring of zeros, which is the 3x3 convolution's zero
// padding. The tap (dy, dx) of a 3x3 convolution is then the constant offset
// dy (Wl + 2) + dx, so an output tile of 128 consecutive positions reads, for
// every tap, 128 consecutive input positions: one contiguous span of the
// input holds the operands of all nine taps. Channels are stored in chunks
// of eight, [C / 8][Qp][8] bf16 (Qp = the positions rounded up to 32), so a
// chunk's span is one contiguous run of 16-byte rows: exactly the K-major
// core-matrix layout (8 positions x 8 channels = 128 contiguous bytes) the
// MMAs read, copied by TMA as one box of 512-byte rows (32 positions each).
//
//   k_conv_tc<0>  3x3 convolution + bias + ReLU as an implicit GEMM
//                 (M = positions, N = output channels, K = 9 x input
//                 channels). A block takes R x 128 positions and NT output
//                 channels. Per K step of 16 input channels one thread issues
//                 TMA copies of the input span (one box per 8-channel chunk,
//                 starting at the 32-position row at or before the span) and
//                 of the step's packed weights into a pipeline stage; another
//                 issues tcgen05.mma (M 128, N NT, K 16) for the nine taps x R
//                 row groups with shared-memory descriptors offset by the tap's
//                 shift; tcgen05.commit frees the stage when its MMAs are
//                 done. The four warps then read the accumulators back
//                 (tcgen05.ld), add the bias, apply ReLU and store bf16, with
//                 zeros on the border ring, one 16-byte store per chunk.
//   k_conv_tc<1>  the output layer: the 1x1 convolution of d0 (32
//                 channels), plus the base (the input views warped to the
//                 output eyes by warp.cu's k_warp_views, RGB / 255)
//                 and the bias, clamped, scaled to 255, rounded half to even,
//                 written as RGBA8 output views.
//   k_pack_w      weights [cout][taps][cin] -> the per-K-step stage images
//                 [n tile][K step][tap][2][NT][8] the MMAs read.
//   k_avgpool2, k_recon_in   pooling and the input packing, between chunked
//                 bordered tensors (interiors only; the borders stay zero).
// The up path needs no concatenation: the last layer of each lower level
// writes its output 2x upsampled (nearest) into a tensor of the next level's
// size, and the next layer reads its first channels from that tensor (map a)
// and the skip channels from the encoder's tensor (map b).
//   k_to_chunked, k_from_chunked   plain NHWC <-> chunked bordered (test hook).
//
// Every wait (mbarrier phases) gives up after 2e9 SM cycles (about one
// second): the block records
// the failure in a status word, waits (again bounded) for its own copies and
// MMAs in flight, frees its tensor memory and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <utility>
#include <vector>

#include "objects.h"

namespace lfdpr {
namespace {

// ---------------------------------------------------------------------------
// tcgen05 / TMA / mbarrier building blocks (inline PTX)
// ---------------------------------------------------------------------------
namespace tc {

// A wait gives up after this many SM clock cycles (about one second).
constexpr long long kWaitCycles = 2000000000ll;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return uint32_t(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ bool try_wait(uint32_t bar, uint32_t par) {
    uint32_t ok;
    asm volatile("{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
                 : "=r"(ok)
                 : "r"(bar), "r"(par)
                 : "memory");
    return ok != 0;
}

// Wait until the phase of parity `par` of the mbarrier at `bar` completes;
// false after kWaitCycles. The clock is read only once the phase is found
// incomplete.
__device__ __forceinline__ bool wait(uint32_t bar, uint32_t par) {
    if (try_wait(bar, par)) return true;
    const long long t0 = clock64();
    for (;;) {
        if (try_wait(bar, par)) return true;
        if (clock64() - t0 > kWaitCycles) return false;
    }
}

__device__ __forceinline__ void init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}

__device__ __forceinline__ void expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// TMA: one box of a 3-D tensor map at coordinates (x, y, z) -> shared memory.
__device__ __forceinline__ void load_box(uint32_t dst, const CUtensorMap* map, int x, int y, int z, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
}

// Bulk copy of `bytes` (multiple of 16, both addresses 16-byte aligned).
__device__ __forceinline__ void load_bulk(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

// Shared-memory matrix descriptor, no swizzle, K-major: core matrices of 8
// rows x 16 bytes (128 contiguous bytes); `lbo` = byte distance between core
// matrices adjacent in K, `sbo` = between core matrices adjacent in M (N).
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return uint64_t((addr >> 4) & 0x3FFFu) | (uint64_t((lbo >> 4) & 0x3FFFu) << 16) |
           (uint64_t((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: BF16 A and B (K-major), FP32 D, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int m, int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(n >> 3) << 17) | (uint32_t(m >> 4) << 24);
}

// D[tmem] (+)= A[a] B[b]^T; accumulate into D when acc != 0.
__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{ .reg .pred p; setp.ne.b32 p, %4, 0; tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p; }" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

// The mbarrier at `bar` receives one arrival when every MMA this thread has
// issued so far is complete.
__device__ __forceinline__ void commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 16 consecutive FP32 columns of this warp's 32 tensor-memory lanes (one lane
// per thread). The load and its wait are one statement, so no register is
// read before the asynchronous load has written it.
__device__ __forceinline__ void ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 16; i++) v[i] = __uint_as_float(r[i]);
}

// 48 consecutive columns (three loads, one wait).
__device__ __forceinline__ void ld48(uint32_t taddr, float* v) {
    uint32_t r[48];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%48];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%49];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%32,%33,%34,%35,%36,%37,%38,%39,%40,%41,%42,%43,%44,%45,%46,%47}, [%50];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
          "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]), "=r"(r[32]),
          "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]), "=r"(r[40]),
          "=r"(r[41]), "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47])
        : "r"(taddr), "r"(taddr + 16), "r"(taddr + 32)
        : "memory");
#pragma unroll
    for (int i = 0; i < 48; i++) v[i] = __uint_as_float(r[i]);
}

}  // namespace tc

// ---------------------------------------------------------------------------
// The tensor-core layer
// ---------------------------------------------------------------------------

// Warp roles of the persistent layer kernel: warp 0 issues the copies, warp 1
// the MMAs, warps 2-9 drain the accumulators in two column halves (warp w
// reads tensor-memory lanes 32 (w % 4) .. 32 (w % 4) + 31, so each group of
// four covers the 128 rows of a tile).
constexpr int kTcThreads = 320;
constexpr int kEpiWarps = 8;

// Geometry of one tensor-core layer launch (host-computed).
struct TcGeom {
    int Hb, Wb, Q;            // bordered rows, columns, positions Hb Wb
    int taps;                 // 9 (3x3) or 1 (1x1)
    int NT, R;                // output channels per tile; 128-position row groups per tile
    int ksteps;               // K steps of 16 input channels
    int split;                // 8-channel chunks read through map a (the rest through map b)
    int rows, span;           // TMA box rows of 32 positions per chunk; span = 32 rows positions in shared memory
    int Qp;                   // positions per chunk in memory (Q rounded up to 32)
    int stages;               // pipeline depth
    uint32_t a_bytes, b_bytes, stage_bytes;
    uint32_t tmem_cols;       // power of two >= 2 R NT (two accumulator buffers)
    int m_tiles, n_tiles;     // tiles: ceil(Q / 128 R) position tiles x output-channel tiles
    int cout;                 // channels of the bf16 output tensor (3x3 layers)
    int up;                   // 3x3 layers: write the output 2x upsampled (nearest) into a tensor of twice the size
    int Wbo, Qpo;             // that tensor's bordered width and positions per chunk
    int nout, H, W;           // output layer: views written, view size
    int bias_n;               // biases staged in shared memory (<= 256)
    const uint32_t* base;     // output layer: the residual's base, RGBA8 views laid out as the output
};

// A wait that also gives up as soon as another role of the block has given
// up (the abort word in shared memory), and sets that word when it times out.
// `backoff_ns` > 0 sleeps between polls (for waits off the critical path, so
// polling does not compete with the copies for the shared-memory pipe).
__device__ __forceinline__ bool wait_or_abort(uint32_t bar, uint32_t par, uint32_t abort_addr,
                                              unsigned backoff_ns = 0) {
    if (tc::try_wait(bar, par)) return true;
    const long long t0 = clock64();
    for (;;) {
        if (backoff_ns) __nanosleep(backoff_ns);
        if (tc::try_wait(bar, par)) return true;
        uint32_t ab;
        asm volatile("ld.volatile.shared.u32 %0, [%1];" : "=r"(ab) : "r"(abort_addr));
        if (ab) return false;
        if (clock64() - t0 > tc::kWaitCycles) {
            asm volatile("st.volatile.shared.u32 [%0], %1;" ::"r"(abort_addr), "r"(1u));
            return false;
        }
    }
}

constexpr int kMaxStages = 8;

// Shared memory: [stages x (A span: 2 chunks x span x 16 B | B: taps x 2 x NT x 16 B)]
// then the barriers: full[8] +0, empty[8] +64, acc_full[2] +128, acc_empty[2]
// +144, drain +160, tensor-memory address +168, abort word +172; then the
// layer's biases (up to 256 floats) at +1024.
// Tile t (t = blockIdx.x, + gridDim.x, ...) covers positions (t % m_tiles) 128 R
// .. + 128 R - 1 and output channels (t / m_tiles) NT .. + NT - 1; its
// accumulators live in tensor-memory buffer (local tile index) % 2.
template <int EPI, int TAPS, int R>
__global__ void __launch_bounds__(kTcThreads, 1) k_conv_tc(const __grid_constant__ CUtensorMap ma,
                                                           const __grid_constant__ CUtensorMap mb,
                                                           const uint8_t* __restrict__ wpk,
                                                           const float* __restrict__ bias, void* __restrict__ out,
                                                           const TcGeom g, int* __restrict__ status) {
    extern __shared__ uint8_t smem_raw[];
    const uint32_t s0 = (tc::smem_u32(smem_raw) + 1023u) & ~1023u;
    const uint32_t bars = s0 + uint32_t(g.stages) * g.stage_bytes;
    const uint32_t empty = bars + 64, acc_full = bars + 128, acc_empty = bars + 144, drain = bars + 160,
                   slot = bars + 168, abort_w = bars + 172;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int n_tiles = g.m_tiles * g.n_tiles;
    const uint32_t acc_cols = uint32_t(R * g.NT);

    if (tid == 0) {
        for (int s = 0; s < g.stages; s++) {
            tc::init(bars + 8 * s, 1);
            tc::init(empty + 8 * s, 1);
        }
        for (int b = 0; b < 2; b++) {
            tc::init(acc_full + 8 * b, 1);
            tc::init(acc_empty + 8 * b, kEpiWarps);   // one arrival per epilogue warp
        }
        tc::init(drain, 1);
        asm volatile("st.shared.u32 [%0], %1;" ::"r"(abort_w), "r"(0u));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    float* s_bias = reinterpret_cast<float*>(smem_raw + (bars + 1024 - tc::smem_u32(smem_raw)));
    for (int i = tid; i < g.bias_n; i += kTcThreads) s_bias[i] = bias[i];
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot),
                     "r"(g.tmem_cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    uint32_t tmem;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(tmem) : "r"(slot));
    wait_previous_kernel();
    allow_next_kernel();

    if (warp == 0) {
        if (lane == 0) {
            // producer: the block's K steps, tile after tile, into stage kc % stages
            int kc = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
                const int q0 = (t % g.m_tiles) * 128 * R, nt = t / g.m_tiles;
                const int qs = q0 - (TAPS == 9 ? g.Wb + 1 : 0);
                const int y0 = (qs >= 0 ? qs : qs - 31) / 32;   // the 32-position row holding the span's start
                const uint8_t* wsrc = wpk + size_t(nt) * g.ksteps * g.b_bytes;
                for (int ks = 0; ks < g.ksteps; ks++, kc++) {
                    const int s = kc % g.stages;
                    if (kc >= g.stages && !wait_or_abort(empty + 8 * s, uint32_t((kc / g.stages - 1) & 1), abort_w)) {
                        ok = false;
                        break;
                    }
                    const uint32_t a = s0 + uint32_t(s) * g.stage_bytes, b = a + g.a_bytes, full = bars + 8 * s;
                    tc::expect_tx(full, g.a_bytes + g.b_bytes);
                    // both 8-channel chunks of the K step in one box (chunk pairs never straddle the maps)
                    const int c8 = 2 * ks;
                    tc::load_box(a, c8 < g.split ? &ma : &mb, 0, y0, c8 < g.split ? c8 : c8 - g.split, full);
                    tc::load_bulk(b, wsrc + size_t(ks) * g.b_bytes, g.b_bytes, full);
                }
            }
            // the copies issued last on each stage have landed before the block moves on
            for (int k = max(0, kc - g.stages); k < kc; k++)
                tc::wait(bars + 8 * (k % g.stages), uint32_t((k / g.stages) & 1));
            if (!ok) atomicOr(status, 1);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // MMA issuer. Descriptors are built once per stage; taps and row groups
            // move the start address by whole 16-byte units (one position), added to
            // the 14-bit address field (shared addresses stay below 256 KB, so the
            // field never carries).
            const uint32_t idesc = tc::idesc_bf16(128, g.NT);
            uint32_t toff[TAPS];
#pragma unroll
            for (int tp = 0; tp < TAPS; tp++) toff[tp] = TAPS == 9 ? uint32_t((tp / 3) * g.Wb + (tp % 3)) : 0u;
            const uint64_t a_desc0 = tc::sdesc(s0, uint32_t(g.span * 16), 128);
            const uint64_t b_desc0 = tc::sdesc(s0 + g.a_bytes, uint32_t(g.NT * 16), 128);
            const uint32_t b_tap = uint32_t(2 * g.NT);   // 16-byte units between taps' weights
            int kc = 0, it = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < n_tiles && ok; t += gridDim.x, it++) {
                const int q0 = (t % g.m_tiles) * 128 * R;
                const int qs = q0 - (TAPS == 9 ? g.Wb + 1 : 0);
                const uint32_t delta = uint32_t(qs - 32 * ((qs >= 0 ? qs : qs - 31) / 32));   // span start in its first row
                const int buf = it & 1;
                // the epilogue has drained this buffer (its use two tiles ago)
                if (it >= 2 && !wait_or_abort(acc_empty + 8 * buf, uint32_t((it / 2 - 1) & 1), abort_w)) {
                    ok = false;
                    break;
                }
                tc::fence_after();
                const uint32_t dacc = tmem + uint32_t(buf) * acc_cols;
                for (int ks = 0; ks < g.ksteps; ks++, kc++) {
                    const int s = kc % g.stages;
                    if (!wait_or_abort(bars + 8 * s, uint32_t((kc / g.stages) & 1), abort_w)) {
                        ok = false;
                        break;
                    }
                    tc::fence_after();
                    const uint32_t st16 = (uint32_t(s) * g.stage_bytes) >> 4;
                    const uint64_t ad = a_desc0 + st16 + delta, bd = b_desc0 + st16;
#pragma unroll
                    for (int tp = 0; tp < TAPS; tp++)
#pragma unroll
                        for (int r = 0; r < R; r++)
                            tc::mma(dacc + uint32_t(r * g.NT), ad + toff[tp] + uint32_t(r * 128), bd + tp * b_tap, idesc,
                                    uint32_t(ks | tp));
                    tc::commit(empty + 8 * s);
                }
                if (ok) tc::commit(acc_full + 8 * buf);
            }
            // every MMA issued has completed before the block moves on
            tc::commit(drain);
            tc::wait(drain, 0);
            if (!ok) atomicOr(status, 2);
        }
    } else {
        // epilogue warps: group cg drains column half cg of every row group
        const int ew = warp - 2, lq = warp & 3, cg = ew >> 2;   // lane quarter, column group
        int it = 0;
        bool ok = true;
        for (int t = blockIdx.x; t < n_tiles; t += gridDim.x, it++) {
            const int q0 = (t % g.m_tiles) * 128 * R, n0 = (t / g.m_tiles) * g.NT;
            const int buf = it & 1;
            // one lane per warp polls (with backoff); the others wait at the shuffle
            int got = 0;
            if (lane == 0) got = wait_or_abort(acc_full + 8 * buf, uint32_t((it / 2) & 1), abort_w, 128) ? 1 : 0;
            ok = __shfl_sync(0xffffffffu, got, 0) != 0;
            if (!ok) break;
            tc::fence_after();
            const uint32_t trow = tmem + (uint32_t(lq * 32) << 16) + uint32_t(buf) * acc_cols;
#pragma unroll
            for (int r = 0; r < R; r++) {
                const int q = q0 + r * 128 + lq * 32 + lane;
                const int y = q / g.Wb, x = q - y * g.Wb;
                if (EPI == 0) {
                    const bool border = y == 0 || y >= g.Hb - 1 || x == 0 || x == g.Wb - 1;
                    const int half = g.NT >> 1;
                    for (int j = cg * half; j < (cg + 1) * half; j += 16) {
                        float v[16], bv[16];
                        tc::ld16(trow + uint32_t(r * g.NT + j), v);
#pragma unroll
                        for (int i = 0; i < 4; i++)
                            *reinterpret_cast<float4*>(bv + 4 * i) = reinterpret_cast<const float4*>(s_bias + n0 + j)[i];
                        uint4 pk[2];
                        __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(pk);
#pragma unroll
                        for (int i = 0; i < 8; i++) {
                            const float a0 = border ? 0.0f : fmaxf(v[2 * i] + bv[2 * i], 0.0f);
                            const float a1 = border ? 0.0f : fmaxf(v[2 * i + 1] + bv[2 * i + 1], 0.0f);
                            h[i] = __floats2bfloat162_rn(a0, a1);
                        }
                        const int c8 = (n0 + j) / 8;
                        if (!g.up) {
                            if (q < g.Q) {
                                __nv_bfloat16* o = static_cast<__nv_bfloat16*>(out) + (size_t(c8) * g.Qp + q) * 8;
                                *reinterpret_cast<uint4*>(o) = pk[0];
                                *reinterpret_cast<uint4*>(o + size_t(g.Qp) * 8) = pk[1];
                            }
                        } else if (q < g.Q && !border) {
                            // nearest 2x: pixel (y - 1, x - 1) -> the 2x2 block at (2 y - 2, 2 x - 2) of the larger image
                            const size_t qh = size_t(2 * y - 1) * g.Wbo + size_t(2 * x - 1);
                            __nv_bfloat16* o = static_cast<__nv_bfloat16*>(out) + (size_t(c8) * g.Qpo + qh) * 8;
#pragma unroll
                            for (int k = 0; k < 2; k++) {
                                __nv_bfloat16* ok_ = o + size_t(k) * g.Qpo * 8;
                                *reinterpret_cast<uint4*>(ok_) = pk[k];
                                *reinterpret_cast<uint4*>(ok_ + 8) = pk[k];
                                *reinterpret_cast<uint4*>(ok_ + size_t(g.Wbo) * 8) = pk[k];
                                *reinterpret_cast<uint4*>(ok_ + size_t(g.Wbo) * 8 + 8) = pk[k];
                            }
                        }
                    }
                } else {
                    // output views: column o = 3 view + channel; 48-column steps alternate between the groups
                    const int vy = y - 1, vx = x - 1;
                    const bool inside = q < g.Q && vy >= 0 && vy < g.H && vx >= 0 && vx < g.W;
                    uint32_t* views = static_cast<uint32_t*>(out);
                    const size_t npix = size_t(g.H) * g.W, pix = size_t(vy) * g.W + vx;
                    for (int j = cg * 48; j < g.NT; j += 96) {
                        float v[48], bv[48];
                        tc::ld48(trow + uint32_t(r * g.NT + j), v);
#pragma unroll
                        for (int i = 0; i < 12; i++)
                            *reinterpret_cast<float4*>(bv + 4 * i) = reinterpret_cast<const float4*>(s_bias + j)[i];
                        // the base's 16 views at this position, all loads in flight first
                        uint32_t bws[16];
#pragma unroll
                        for (int k = 0; k < 16; k++) {
                            const int view = j / 3 + k;
                            bws[k] = inside && view < g.nout ? __ldg(g.base + size_t(view) * npix + pix) : 0u;
                        }
#pragma unroll
                        for (int k = 0; k < 16; k++) {
                            const int view = j / 3 + k;
                            if (!(inside && view < g.nout)) continue;
                            // the base's RGB / 255, added to the product
                            const uint32_t bw = bws[k];
                            float base[3];
#pragma unroll
                            for (int c = 0; c < 3; c++) base[c] = float((bw >> (8 * c)) & 255u) * (1.0f / 255.0f);
                            // round(clamp(x + base + b, 0, 1) 255), half to even: saturating add, scale, convert
                            const uint32_t r0 = __float2uint_rn(__saturatef((v[3 * k] + base[0]) + bv[3 * k]) * 255.0f);
                            const uint32_t g0 =
                                __float2uint_rn(__saturatef((v[3 * k + 1] + base[1]) + bv[3 * k + 1]) * 255.0f);
                            const uint32_t b0 =
                                __float2uint_rn(__saturatef((v[3 * k + 2] + base[2]) + bv[3 * k + 2]) * 255.0f);
                            views[size_t(view) * npix + pix] = 0xff000000u | r0 | (g0 << 8) | (b0 << 16);
                        }
                    }
                }
            }
            // this warp's reads of the buffer are done
            tc::fence_before();
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(acc_empty + 8 * buf) : "memory");
        }
        if (!ok && lane == 0) atomicOr(status, 4);
    }
    __syncwarp();
    tc::fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(g.tmem_cols));
}

// dst [n_tiles][ksteps][taps][2][NT][8] from src [cout][taps][cin]; rows co >=
// cout are zero (cin % 16 == 0).
__global__ void k_pack_w(const __nv_bfloat16* __restrict__ src, int cout, int taps, int cin, int NT, int n_tiles,
                         __nv_bfloat16* __restrict__ dst) {
    const int ksteps = cin / 16;
    const size_t total = size_t(n_tiles) * ksteps * taps * 2 * NT * 8;
    for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < total; i += size_t(gridDim.x) * blockDim.x) {
        size_t r = i;
        const int e = int(r % 8);
        r /= 8;
        const int n = int(r % NT);
        r /= NT;
        const int c2 = int(r % 2);
        r /= 2;
        const int t = int(r % taps);
        r /= taps;
        const int ks = int(r % ksteps);
        const int ntile = int(r / ksteps);
        const int co = ntile * NT + n, ci = ks * 16 + c2 * 8 + e;
        dst[i] = co < cout ? src[(size_t(co) * taps + t) * cin + ci] : __float2bfloat16_rn(0.0f);
    }
}

// Chunked bordered tensors: channel c of level-image pixel (y, x) (H x W) is
// element ((c / 8) Qp + q) 8 + c % 8 with q = (y + 1) (W + 2) + x + 1 and
// Qp = (H + 2) (W + 2) rounded up to 32.
__host__ __device__ __forceinline__ size_t qpad(int H, int W) { return (size_t(H + 2) * (W + 2) + 31) / 32 * 32; }
__device__ __forceinline__ size_t bpos(int y, int x, int W) { return size_t(y + 1) * (W + 2) + (x + 1); }

__device__ __forceinline__ void bf16x8_to_f32(const uint4& v, float* f) {
    const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&v);
#pragma unroll
    for (int e = 0; e < 4; e++) {
        const float2 t = __bfloat1622float2(h[e]);
        f[2 * e] = t.x;
        f[2 * e + 1] = t.y;
    }
}
__device__ __forceinline__ uint4 f32_to_bf16x8(const float* f) {
    uint4 o;
    __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(&o);
#pragma unroll
    for (int e = 0; e < 4; e++) h[e] = __floats2bfloat162_rn(f[2 * e], f[2 * e + 1]);
    return o;
}

// out (level H/2 x W/2) = mean of 2x2 blocks of in (level H x W); C % 8 == 0.
// One thread per (chunk, output pixel), pixels fastest.
__global__ void k_avgpool2(const __nv_bfloat16* __restrict__ in, int H, int W, int C, __nv_bfloat16* __restrict__ out) {
    wait_previous_kernel();
    allow_next_kernel();
    const int Ho = H / 2, Wo = W / 2;
    const size_t npx = size_t(Ho) * Wo, total = npx * (C / 8), qi = qpad(H, W), qo = qpad(Ho, Wo);
    for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < total; i += size_t(gridDim.x) * blockDim.x) {
        const int c8 = int(i / npx);
        const size_t p = i - c8 * npx;
        const int xo = int(p % Wo), yo = int(p / Wo);
        const __nv_bfloat16* src = in + size_t(c8) * qi * 8;
        float s[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int q = 0; q < 4; q++) {
            float f[8];
            bf16x8_to_f32(*reinterpret_cast<const uint4*>(src + bpos(2 * yo + (q >> 1), 2 * xo + (q & 1), W) * 8), f);
#pragma unroll
            for (int e = 0; e < 8; e++) s[e] += f[e];
        }
#pragma unroll
        for (int e = 0; e < 8; e++) s[e] *= 0.25f;
        *reinterpret_cast<uint4*>(out + (size_t(c8) * qo + bpos(yo, xo, Wo)) * 8) = f32_to_bf16x8(s);
    }
}

// x0 (level Hp x Wp, 48 channels): channel 3 j + c = channel c of input view
// j / 255 for j < nin (nin <= 16), zero elsewhere and outside the H x W views.
// One thread per pixel: its nin RGBA8 words, six 16-byte chunk stores.
__global__ void k_recon_in(const uint8_t* __restrict__ views, int nin, int H, int W, int Hp, int Wp,
                           __nv_bfloat16* __restrict__ x0) {
    allow_next_kernel();   // launched plainly: it waits for everything before it
    const size_t total = size_t(Hp) * Wp, npix = size_t(H) * W, qp = qpad(Hp, Wp);
    for (size_t p = size_t(blockIdx.x) * blockDim.x + threadIdx.x; p < total; p += size_t(gridDim.x) * blockDim.x) {
        const int x = int(p % Wp), y = int(p / Wp);
        float v[48];
#pragma unroll
        for (int j = 0; j < 16; j++) {
            uint32_t w = 0u;
            if (j < nin && x < W && y < H) w = __ldg(reinterpret_cast<const uint32_t*>(views) + size_t(j) * npix + size_t(y) * W + x);
#pragma unroll
            for (int c = 0; c < 3; c++) v[3 * j + c] = float((w >> (8 * c)) & 255u) * (1.0f / 255.0f);
        }
        const size_t q = bpos(y, x, Wp);
#pragma unroll
        for (int g = 0; g < 6; g++) *reinterpret_cast<uint4*>(x0 + (size_t(g) * qp + q) * 8) = f32_to_bf16x8(v + 8 * g);
    }
}

// Plain NHWC [H][W][C] <-> chunked bordered (test hook; C % 8 == 0).
__global__ void k_to_chunked(const __nv_bfloat16* __restrict__ in, int H, int W, int C, __nv_bfloat16* __restrict__ out) {
    const size_t npx = size_t(H) * W, total = npx * (C / 8), qp = qpad(H, W);
    for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < total; i += size_t(gridDim.x) * blockDim.x) {
        const int c8 = int(i / npx);
        const size_t p = i - c8 * npx;
        *reinterpret_cast<uint4*>(out + (size_t(c8) * qp + bpos(int(p / W), int(p % W), W)) * 8) =
            *reinterpret_cast<const uint4*>(in + p * C + 8 * c8);
    }
}
__global__ void k_from_chunked(const __nv_bfloat16* __restrict__ in, int H, int W, int C, __nv_bfloat16* __restrict__ out) {
    const size_t npx = size_t(H) * W, total = npx * (C / 8), qp = qpad(H, W);
    for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < total; i += size_t(gridDim.x) * blockDim.x) {
        const int c8 = int(i / npx);
        const size_t p = i - c8 * npx;
        *reinterpret_cast<uint4*>(out + p * C + 8 * c8) =
            *reinterpret_cast<const uint4*>(in + (size_t(c8) * qp + bpos(int(p / W), int(p % W), W)) * 8);
    }
}

// ---------------------------------------------------------------------------
// Host side of the tensor-core layers
// ---------------------------------------------------------------------------

constexpr uint32_t kTcSmemMax = 227 * 1024;

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        cudaDriverEntryPointQueryResult q;
        void* p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// 3-D map over a chunked bordered tensor [C / 8][Qp][8] bf16 seen as
// (256 elements = 32 positions x 8 channels, Qp / 32 rows, C / 8 chunks):
// boxes of `rows` 512-byte rows of two consecutive chunks.
cudaError_t make_map(CUtensorMap* m, const void* base, int C, size_t Qp, int rows) {
    auto enc = tensor_map_encoder();
    if (!enc) return cudaErrorNotSupported;
    if ((reinterpret_cast<uintptr_t>(base) & 15) || C % 8 || Qp % 32 || rows < 1 || rows > 256)
        return cudaErrorInvalidValue;
    const cuuint64_t dims[3] = {256, cuuint64_t(Qp / 32), cuuint64_t(C / 8)};
    const cuuint64_t strides[2] = {512, cuuint64_t(Qp) * 16};
    const cuuint32_t box[3] = {256, cuuint32_t(rows), 2}, es[3] = {1, 1, 1};
    const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box, es,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

uint32_t pow2_cols(int n) {
    uint32_t c = 32;
    while (c < uint32_t(n)) c <<= 1;
    return c;
}

// Geometry of a layer over the bordered level image Hl x Wl: cin = cin_a +
// cin_b input channels (map a, then map b), NT output channels per block, R
// row groups of 128 positions per block.
TcGeom tc_geom(int Hl, int Wl, int cin_a, int cin_b, int taps, int NT, int R, int n_tiles, int cout) {
    TcGeom g{};
    g.Hb = Hl + 2;
    g.Wb = Wl + 2;
    g.Q = g.Hb * g.Wb;
    g.taps = taps;
    g.NT = NT;
    g.R = R;
    g.ksteps = (cin_a + cin_b) / 16;
    g.split = cin_a / 8;
    g.Qp = (g.Q + 31) / 32 * 32;
    // the span plus up to 31 positions before it in its first 32-position row
    const int L = 128 * R + (taps == 9 ? 2 * g.Wb + 2 : 0);
    g.rows = (L + 31 + 31) / 32;
    g.span = 32 * g.rows;
    g.a_bytes = uint32_t(2 * g.span * 16);
    g.b_bytes = uint32_t(taps * 2 * NT * 16);
    g.stage_bytes = (g.a_bytes + g.b_bytes + 1023u) & ~1023u;
    // one block per SM, as many stages as fit
    g.stages = int(std::min<uint32_t>(uint32_t(kMaxStages), (kTcSmemMax - 3072u) / g.stage_bytes));
    g.tmem_cols = pow2_cols(2 * R * NT);
    g.m_tiles = (g.Q + 128 * R - 1) / (128 * R);
    g.n_tiles = n_tiles;
    g.cout = cout;
    g.bias_n = n_tiles * NT;
    return g;
}

// Shared memory of one SM (bytes), queried once per process.
size_t smem_per_sm() {
    static int v = 0;
    if (!v) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess || v <= 0)
            v = 228 * 1024;
    }
    return size_t(v);
}

// Dynamic shared memory of a block: the stages, the barriers, the 1024-byte
// alignment slack, and more than half of the SM's, so that one block holds
// an SM (and its tensor memory) at a time.
size_t tc_smem(const TcGeom& g) {
    return std::max(size_t(g.stages) * g.stage_bytes + 2048 + 1024, smem_per_sm() / 2 + 1024);
}

int sm_count_cached() {
    static int v = 0;
    if (!v) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 1;
    }
    return v;
}

bool tc_valid(const TcGeom& g) {
    return g.stages >= 2 && g.ksteps >= 1 && g.NT % 16 == 0 && g.NT >= 16 && g.NT <= 256 && g.tmem_cols <= 512 &&
           (g.taps == 9 || g.taps == 1) && g.split % 2 == 0 && g.rows <= 256 && g.m_tiles >= 1 && g.n_tiles >= 1 &&
           g.bias_n >= 1 && g.bias_n <= 256 && (g.taps == 1 || (g.NT / 2) % 16 == 0) && tc_smem(g) <= kTcSmemMax;
}

// Each layer is launched as a programmatic dependent of the kernel before it
// (launch_after_previous): its blocks set up their barriers, tensor memory
// and biases, then wait for that kernel in wait_previous_kernel().
cudaError_t launch_tc(int epi, const TcGeom& g, const CUtensorMap& ma, const CUtensorMap& mb, const void* wpk,
                      const float* bias, void* out, int* status, cudaStream_t s) {
    if (!tc_valid(g)) return cudaErrorInvalidValue;
    static bool attrs[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!attrs[dev]) {
        const void* fns[4] = {reinterpret_cast<const void*>(k_conv_tc<1, 1, 1>), reinterpret_cast<const void*>(k_conv_tc<0, 9, 1>),
                              reinterpret_cast<const void*>(k_conv_tc<0, 9, 2>), reinterpret_cast<const void*>(k_conv_tc<0, 9, 4>)};
        for (const void* f : fns) {
            const cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kTcSmemMax));
            if (e != cudaSuccess) return e;
        }
        attrs[dev] = true;
    }
    const int grid = std::min(g.m_tiles * g.n_tiles, sm_count_cached());
    const size_t smem = tc_smem(g);
    const uint8_t* w = static_cast<const uint8_t*>(wpk);
    if (epi == 1 && g.taps == 1 && g.R == 1)
        return launch_after_previous(k_conv_tc<1, 1, 1>, grid, kTcThreads, smem, s, ma, mb, w, bias, out, g, status);
    if (epi == 0 && g.taps == 9 && g.R == 1)
        return launch_after_previous(k_conv_tc<0, 9, 1>, grid, kTcThreads, smem, s, ma, mb, w, bias, out, g, status);
    if (epi == 0 && g.taps == 9 && g.R == 2)
        return launch_after_previous(k_conv_tc<0, 9, 2>, grid, kTcThreads, smem, s, ma, mb, w, bias, out, g, status);
    if (epi == 0 && g.taps == 9 && g.R == 4)
        return launch_after_previous(k_conv_tc<0, 9, 4>, grid, kTcThreads, smem, s, ma, mb, w, bias, out, g, status);
    return cudaErrorInvalidValue;
}

cudaError_t launch_pack(const __nv_bfloat16* src, int cout, int taps, int cin, int NT, int n_tiles, __nv_bfloat16* dst,
                        cudaStream_t s) {
    k_pack_w<<<256, 256, 0, s>>>(src, cout, taps, cin, NT, n_tiles, dst);
    return cudaGetLastError();
}

// Output channels and row groups per tile of a 3x3 layer: 128, 64 or 32 channels
// (wider tiles re-read each input span for fewer output channels);
// the most row groups (two accumulator buffers of R NT <= 256 columns each)
// that still give every SM two tiles or more.
void pick_tile(int Hl, int Wl, int cout, int sm_count, int& NT, int& R) {
    NT = cout % 128 == 0 ? 128 : cout % 64 == 0 ? 64 : 32;
    const int64_t Q = int64_t(Hl + 2) * (Wl + 2);
    R = 1;
    for (int r : {4, 2}) {
        if (r * NT > 128) continue;
        if ((Q + 128 * r - 1) / (128 * r) * (cout / NT) >= 2 * sm_count) {
            R = r;
            break;
        }
    }
}

}  // namespace
}  // namespace lfdpr

// ---------------------------------------------------------------------------
// The network (host side)
// ---------------------------------------------------------------------------

using namespace lfdpr;

namespace {

struct ConvSpec {
    int cin, cout, level;   // input channels (padded), output channels, resolution level 0..3
};
// The U-Net's 3x3 layers in order (two per level down, a bottleneck pair, two
// per level up; up-path inputs are [upsampled, skip] concatenations).
const ConvSpec kLayers[14] = {{48, 32, 0},  {32, 32, 0},   {32, 64, 1},   {64, 64, 1},   {64, 128, 2},
                              {128, 128, 2}, {128, 256, 3}, {256, 256, 3}, {384, 128, 2}, {128, 128, 2},
                              {192, 64, 1},  {64, 64, 1},   {96, 32, 0},   {32, 32, 0}};

}  // namespace

struct lfdpr_recon {
    int W = 0, H = 0, Wp = 0, Hp = 0, nin = 0, nout = 0, sm_count = 1;
    __nv_bfloat16* w = nullptr;       // packed 3x3 weights, layer by layer
    float* b = nullptr;               // all 3x3 biases
    __nv_bfloat16* w_out = nullptr;   // packed output layer: 32 (1x1 weights) x NT_out
    float* b_out = nullptr;           // [NT_out] (zero past 3 nout)
    int* status = nullptr;            // device: failed waits (bit 0 copies, 1 MMA, 2 epilogue)
    int64_t w_off[14] = {}, b_off[14] = {};
    TcGeom geom[14] = {}, geom_out = {};
    CUtensorMap in_map[14], in_map_b[14], out_d0;
    uint8_t* warp = nullptr;          // [nout][H][W][4] the input views warped to the output eyes (RGBA8)
    cudaStream_t side = nullptr;      // the warp runs here, beside the network's layers
    cudaEvent_t fork = nullptr, join = nullptr;
    __nv_bfloat16* act = nullptr;     // activation arena (chunked bordered tensors)
    // encoder e*, pooled p*, bottleneck ba, upsampled U* (written by layers 7, 9, 11), decoder d*
    __nv_bfloat16 *x0, *e0a, *e0, *p1, *e1a, *e1, *p2, *e2a, *e2, *p3, *ba, *U2, *d2a, *U1, *d1a, *U0, *d0a, *d0;
};

namespace {

void free_recon(lfdpr_recon* r) {
    if (!r) return;
    dev_free(r->w);
    dev_free(r->b);
    dev_free(r->w_out);
    dev_free(r->b_out);
    dev_free(r->status);
    dev_free(r->warp);
    dev_free(r->act);
    if (r->fork) cudaEventDestroy(r->fork);
    if (r->join) cudaEventDestroy(r->join);
    if (r->side) cudaStreamDestroy(r->side);
    delete r;
}

// Output channels of the output layer's blocks: 3 nout padded to a multiple of 48.
int out_nt(int nout) { return (3 * nout + 47) / 48 * 48; }

}  // namespace

extern "C" {

int64_t lfdpr_recon_weight_count(int32_t in_views) {
    int64_t n = 0;
    for (const auto& L : kLayers) n += int64_t(L.cout) * 9 * L.cin;
    return n + int64_t(3 * 4 * in_views) * 32;
}

int64_t lfdpr_recon_bias_count(int32_t in_views) {
    int64_t n = 0;
    for (const auto& L : kLayers) n += L.cout;
    return n + 3 * 4 * in_views;
}

lfdpr_status lfdpr_create_recon(int32_t view_w, int32_t view_h, int32_t in_views, const uint16_t* weights_bf16,
                                int64_t n_weights, const float* biases, int64_t n_biases, lfdpr_recon** out) {
    lfdpr::g_last_error[0] = 0;
    if (!out || !weights_bf16 || !biases) return fail(LFDPR_EINVAL, "create_recon: null argument");
    *out = nullptr;
    if (in_views < 2 || in_views > 16 || (in_views & 1))
        return fail(LFDPR_EINVAL, "create_recon: in_views must be even, in [2, 16]");
    if (view_w < 8 || view_h < 8 || view_w > kMaxWarpWidth || view_h > 4096)
        return fail(LFDPR_EINVAL, "create_recon: views must be 8..%d pixels wide, 8..4096 high", kMaxWarpWidth);
    if (n_weights != lfdpr_recon_weight_count(in_views) || n_biases != lfdpr_recon_bias_count(in_views))
        return fail(LFDPR_EINVAL, "create_recon: expected %lld weights and %lld biases",
                    (long long)lfdpr_recon_weight_count(in_views), (long long)lfdpr_recon_bias_count(in_views));
    if (!tensor_map_encoder()) return fail(LFDPR_ECUDA, "create_recon: the driver has no tensor-map encoder");
    lfdpr_recon* r = new (std::nothrow) lfdpr_recon();
    if (!r) return fail(LFDPR_ENOMEM, "host allocation failed");
    r->W = view_w;
    r->H = view_h;
    r->Wp = (view_w + 7) / 8 * 8;
    r->Hp = (view_h + 7) / 8 * 8;
    r->nin = in_views;
    r->nout = 4 * in_views;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&r->sm_count, cudaDevAttrMultiProcessorCount, dev);
    int64_t wo = 0, bo = 0;
    for (int l = 0; l < 14; l++) {
        r->w_off[l] = wo;
        r->b_off[l] = bo;
        wo += int64_t(kLayers[l].cout) * 9 * kLayers[l].cin;
        bo += kLayers[l].cout;
    }
    // activation arena: every bordered tensor of the forward pass, 256-byte aligned
    int64_t Ql[4];   // positions per chunk of each level
    for (int l = 0; l < 4; l++) Ql[l] = int64_t(qpad(r->Hp >> l, r->Wp >> l));
    constexpr int kTensors = 18;
    const int64_t sizes[kTensors] = {Ql[0] * 48,  Ql[0] * 32,  Ql[0] * 32, Ql[1] * 32, Ql[1] * 64,  Ql[1] * 64,
                                     Ql[2] * 64,  Ql[2] * 128, Ql[2] * 128, Ql[3] * 128, Ql[3] * 256, Ql[2] * 256,
                                     Ql[2] * 128, Ql[1] * 128, Ql[1] * 64,  Ql[0] * 64,  Ql[0] * 32,  Ql[0] * 32};
    int64_t offs[kTensors], total = 0;
    for (int k = 0; k < kTensors; k++) {
        offs[k] = total;
        total += (sizes[k] + 127) / 128 * 128;
    }
    const int ntout = out_nt(r->nout), no3 = 3 * r->nout, ko = 32;
    cudaError_t e;
    const int64_t nw3 = wo, nb3 = bo;
    uint16_t* w_raw = nullptr;   // device staging of the 3x3 blob before packing
    uint16_t* wout_raw = nullptr;
    if ((e = dev_malloc(&r->w, 2 * nw3)) != cudaSuccess || (e = dev_malloc(&r->b, 4 * nb3)) != cudaSuccess ||
        (e = dev_malloc(&r->w_out, 2 * int64_t(ntout) * ko)) != cudaSuccess ||
        (e = dev_malloc(&r->warp, 4 * int64_t(r->nout) * r->W * r->H)) != cudaSuccess ||
        (e = dev_malloc(&r->b_out, 4 * int64_t(ntout))) != cudaSuccess ||
        (e = dev_malloc(&r->status, sizeof(int))) != cudaSuccess || (e = dev_malloc(&r->act, 2 * total)) != cudaSuccess ||
        (e = dev_malloc(&w_raw, 2 * nw3)) != cudaSuccess ||
        (e = dev_malloc(&wout_raw, 2 * int64_t(no3) * ko)) != cudaSuccess) {
        dev_free(w_raw);
        dev_free(wout_raw);
        free_recon(r);
        return cuda_fail(e, "create_recon: allocation");
    }
    if ((e = cudaStreamCreateWithFlags(&r->side, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&r->fork, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&r->join, cudaEventDisableTiming)) != cudaSuccess) {
        dev_free(w_raw);
        dev_free(wout_raw);
        free_recon(r);
        return cuda_fail(e, "create_recon: stream");
    }
    __nv_bfloat16** bufs[kTensors] = {&r->x0,  &r->e0a, &r->e0, &r->p1, &r->e1a, &r->e1,  &r->p2,  &r->e2a, &r->e2,
                                      &r->p3,  &r->ba,  &r->U2, &r->d2a, &r->U1, &r->d1a, &r->U0, &r->d0a, &r->d0};
    for (int k = 0; k < kTensors; k++) *bufs[k] = r->act + offs[k];
    // the output layer's 32 weights per output channel (the base is added in
    // its epilogue)
    std::vector<uint16_t> wout(size_t(no3) * ko, 0);
    for (int o = 0; o < no3; o++)
        for (int k = 0; k < 32; k++) wout[size_t(o) * ko + k] = weights_bf16[nw3 + int64_t(o) * 32 + k];
    std::vector<float> bout(ntout, 0.0f);
    for (int o = 0; o < no3; o++) bout[o] = biases[nb3 + o];
    // layer geometry and packed weights
    for (int l = 0; l < 14; l++) {
        const ConvSpec& L = kLayers[l];
        const int Hl = r->Hp >> L.level, Wl = r->Wp >> L.level;
        int NT, R;
        pick_tile(Hl, Wl, L.cout, r->sm_count, NT, R);
        // layers 8, 10, 12 read [upsampled (map a) | skip (map b)]
        const int cin_b = (l == 8 || l == 10 || l == 12) ? L.cin / 3 : 0;
        r->geom[l] = tc_geom(Hl, Wl, L.cin - cin_b, cin_b, 9, NT, R, L.cout / NT, L.cout);
        if (l == 7 || l == 9 || l == 11) {   // write 2x upsampled into the next level's tensor
            r->geom[l].up = 1;
            r->geom[l].Wbo = 2 * Wl + 2;
            r->geom[l].Qpo = int(qpad(2 * Hl, 2 * Wl));
        }
    }
    r->geom_out = tc_geom(r->Hp, r->Wp, 32, 0, 1, ntout, 1, 1, 0);
    r->geom_out.base = reinterpret_cast<const uint32_t*>(r->warp);
    r->geom_out.nout = r->nout;
    r->geom_out.H = r->H;
    r->geom_out.W = r->W;
    const __nv_bfloat16* conv_in[14] = {r->x0, r->e0a, r->p1, r->e1a, r->p2, r->e2a, r->p3,
                                        r->ba, r->U2,  r->d2a, r->U1, r->d1a, r->U0, r->d0a};
    const __nv_bfloat16* conv_skip[14] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr,
                                          nullptr, r->e2,  nullptr, r->e1,  nullptr, r->e0,  nullptr};
    bool maps_ok = true;
    for (int l = 0; l < 14 && maps_ok; l++) {
        const TcGeom& g = r->geom[l];
        const int cin_a = 8 * g.split;
        maps_ok = tc_valid(g) && make_map(&r->in_map[l], conv_in[l], cin_a, g.Qp, g.rows) == cudaSuccess;
        if (maps_ok && conv_skip[l])
            maps_ok = make_map(&r->in_map_b[l], conv_skip[l], kLayers[l].cin - cin_a, g.Qp, g.rows) == cudaSuccess;
        else
            r->in_map_b[l] = r->in_map[l];
    }
    maps_ok = maps_ok && tc_valid(r->geom_out) &&
              make_map(&r->out_d0, r->d0, 32, r->geom_out.Qp, r->geom_out.rows) == cudaSuccess;
    if (!maps_ok) {
        dev_free(w_raw);
        dev_free(wout_raw);
        free_recon(r);
        return fail(LFDPR_EINVAL, "create_recon: no tensor-core layout for %dx%d views", view_w, view_h);
    }
    if ((e = cudaMemcpy(w_raw, weights_bf16, 2 * nw3, cudaMemcpyHostToDevice)) == cudaSuccess &&
        (e = cudaMemcpy(wout_raw, wout.data(), 2 * wout.size(), cudaMemcpyHostToDevice)) == cudaSuccess &&
        (e = cudaMemcpy(r->b, biases, 4 * nb3, cudaMemcpyHostToDevice)) == cudaSuccess &&
        (e = cudaMemcpy(r->b_out, bout.data(), 4 * bout.size(), cudaMemcpyHostToDevice)) == cudaSuccess &&
        (e = cudaMemset(r->act, 0, 2 * total)) == cudaSuccess && (e = cudaMemset(r->status, 0, sizeof(int))) == cudaSuccess) {
        for (int l = 0; l < 14 && e == cudaSuccess; l++)
            e = launch_pack(reinterpret_cast<const __nv_bfloat16*>(w_raw) + r->w_off[l], kLayers[l].cout, 9,
                            kLayers[l].cin, r->geom[l].NT, r->geom[l].n_tiles, r->w + r->w_off[l], 0);
        if (e == cudaSuccess)
            e = launch_pack(reinterpret_cast<const __nv_bfloat16*>(wout_raw), no3, 1, ko, ntout, 1, r->w_out, 0);
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
    }
    dev_free(w_raw);
    dev_free(wout_raw);
    if (e != cudaSuccess) {
        free_recon(r);
        return cuda_fail(e, "create_recon: upload");
    }
    *out = r;
    return LFDPR_OK;
}

lfdpr_status lfdpr_destroy_recon(lfdpr_recon* r) {
    lfdpr::g_last_error[0] = 0;
    if (!r) return fail(LFDPR_EINVAL, "destroy_recon: null");
    free_recon(r);
    return LFDPR_OK;
}

lfdpr_status lfdpr_recon_forward(lfdpr_recon* r, const uint8_t* in_views, const uint64_t* in_keys,
                                 const float* in_eyes, const float* out_eyes, float pixels_per_unit,
                                 uint8_t* out_views, void* stream) {
    lfdpr::g_last_error[0] = 0;
    if (!r || !in_views || !in_keys || !in_eyes || !out_eyes || !out_views)
        return fail(LFDPR_EINVAL, "recon_forward: null argument");
    if (!(pixels_per_unit > 0.0f) || !std::isfinite(pixels_per_unit))
        return fail(LFDPR_EINVAL, "recon_forward: pixels_per_unit must be positive and finite");
    if ((reinterpret_cast<uintptr_t>(in_views) & 3u) || (reinterpret_cast<uintptr_t>(out_views) & 3u) ||
        (reinterpret_cast<uintptr_t>(in_keys) & 7u) || (reinterpret_cast<uintptr_t>(in_eyes) & 3u) ||
        (reinterpret_cast<uintptr_t>(out_eyes) & 3u))
        return fail(LFDPR_EINVAL, "recon_forward: views and eyes must be 4-byte aligned, keys 8-byte aligned");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int H0 = r->Hp, W0 = r->Wp, sm = r->sm_count;
    __nv_bfloat16* conv_out[14] = {r->e0a, r->e0, r->e1a, r->e1, r->e2a, r->e2, r->ba,
                                   r->U2,  r->d2a, r->U1, r->d1a, r->U0, r->d0a, r->d0};
    auto conv = [&](int l) {
        return launch_tc(0, r->geom[l], r->in_map[l], r->in_map_b[l], r->w + r->w_off[l], r->b + r->b_off[l],
                         conv_out[l], r->status, s);
    };
    auto pool = [&](const __nv_bfloat16* in, int H, int W, int C, __nv_bfloat16* o) {
        return launch_after_previous(k_avgpool2, sm * 8, 256, 0, s, in, H, W, C, o);
    };
#define CKR(call, what)                                      \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) return cuda_fail(e_, what);   \
    } while (0)
    k_recon_in<<<sm * 8, 256, 0, s>>>(in_views, r->nin, r->H, r->W, H0, W0, r->x0);
    CKR(cudaGetLastError(), "launch k_recon_in");
    // the residual's base: the input views warped to the output eyes, on the
    // side stream while the layers run (SMs the layers leave idle take it)
    CKR(cudaEventRecord(r->fork, s), "recon_forward: fork");
    CKR(cudaStreamWaitEvent(r->side, r->fork, 0), "recon_forward: fork");
    CKR(launch_warp_views(in_views, in_keys, in_eyes, r->nin, out_eyes, r->nout, r->W, r->H, pixels_per_unit,
                          r->warp, r->side),
        "launch k_warp_views");
    CKR(cudaEventRecord(r->join, r->side), "recon_forward: join");

    CKR(conv(0), "conv 0");
    CKR(conv(1), "conv 1");
    CKR(pool(r->e0, H0, W0, 32, r->p1), "pool 1");
    CKR(conv(2), "conv 2");
    CKR(conv(3), "conv 3");
    CKR(pool(r->e1, H0 / 2, W0 / 2, 64, r->p2), "pool 2");
    CKR(conv(4), "conv 4");
    CKR(conv(5), "conv 5");
    CKR(pool(r->e2, H0 / 4, W0 / 4, 128, r->p3), "pool 3");
    CKR(conv(6), "conv 6");
    CKR(conv(7), "conv 7");
    CKR(conv(8), "conv 8");
    CKR(conv(9), "conv 9");
    CKR(conv(10), "conv 10");
    CKR(conv(11), "conv 11");
    CKR(conv(12), "conv 12");
    CKR(conv(13), "conv 13");
    CKR(cudaStreamWaitEvent(s, r->join, 0), "recon_forward: join");
    CKR(launch_tc(1, r->geom_out, r->out_d0, r->out_d0, r->w_out, r->b_out, out_views, r->status, s),
        "output layer");
#undef CKR
    return LFDPR_OK;
}

lfdpr_status lfdpr_recon_run(lfdpr_recon* r, const lfdpr_display* src, lfdpr_display* dst, void* stream) {
    lfdpr::g_last_error[0] = 0;
    if (!r || !src || !dst) return fail(LFDPR_EINVAL, "recon_run: null argument");
    if (src->dc.nr != r->nin || src->dc.W != r->W || src->dc.H != r->H)
        return fail(LFDPR_EINVAL, "recon_run: source display must render %d views of %dx%d", r->nin, r->W, r->H);
    if (dst->dc.nr != r->nout || dst->dc.W != r->W || dst->dc.H != r->H)
        return fail(LFDPR_EINVAL, "recon_run: target display must hold %d views of %dx%d", r->nout, r->W, r->H);
    return lfdpr_recon_forward(r, src->views, src->keys, src->d_ex, dst->d_ex, src->dc.ipw, dst->views, stream);
}

lfdpr_status lfdpr_recon_status(lfdpr_recon* r, int32_t* flags) {
    lfdpr::g_last_error[0] = 0;
    if (!r || !flags) return fail(LFDPR_EINVAL, "recon_status: null argument");
    int v = 0;
    cudaError_t e = cudaMemcpy(&v, r->status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(r->status, 0, sizeof(int));
    if (e != cudaSuccess) return cuda_fail(e, "recon_status");
    *flags = v;
    return LFDPR_OK;
}

lfdpr_status lfdpr_conv3x3_bf16(const void* in, int32_t H, int32_t W, int32_t cin, const void* wgt, const float* bias,
                                void* out, int32_t cout, int32_t* status, void* stream) {
    lfdpr::g_last_error[0] = 0;
    if (!in || !wgt || !bias || !out || !status) return fail(LFDPR_EINVAL, "conv3x3: null argument");
    if (H < 1 || W < 1 || H > 8192 || W > 8192 || cin < 16 || cin % 16 || cin > 512 || cout < 32 || cout % 32 ||
        cout > 256)
        return fail(LFDPR_EINVAL, "conv3x3: need cin %% 16 == 0 (<= 512), cout %% 32 == 0 (<= 256)");
    if ((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(out) | reinterpret_cast<uintptr_t>(wgt)) & 15)
        return fail(LFDPR_EINVAL, "conv3x3: buffers must be 16-byte aligned");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int NT, R;
    pick_tile(H, W, cout, sms, NT, R);
    const TcGeom g = tc_geom(H, W, cin, 0, 9, NT, R, cout / NT, cout);
    if (!tc_valid(g)) return fail(LFDPR_EINVAL, "conv3x3: no tensor-core layout for a %d-wide image", W);
    // chunked bordered copies of the input and output, and the packed weights
    const size_t qp = qpad(H, W);
    __nv_bfloat16 *ci = nullptr, *co = nullptr, *wpk = nullptr;
    cudaError_t e = dev_malloc_async(&ci, 2 * qp * cin, s);
    if (e == cudaSuccess) e = dev_malloc_async(&co, 2 * qp * cout, s);
    if (e == cudaSuccess) e = dev_malloc_async(&wpk, size_t(2) * cout * 9 * cin, s);
    CUtensorMap m;
    if (e == cudaSuccess) e = cudaMemsetAsync(ci, 0, 2 * qp * cin, s);
    if (e == cudaSuccess) e = make_map(&m, ci, cin, qp, g.rows);
    if (e == cudaSuccess) {
        k_to_chunked<<<sms * 8, 256, 0, s>>>(static_cast<const __nv_bfloat16*>(in), H, W, cin, ci);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = launch_pack(static_cast<const __nv_bfloat16*>(wgt), cout, 9, cin, NT, cout / NT, wpk, s);
    if (e == cudaSuccess) e = launch_tc(0, g, m, m, wpk, bias, co, reinterpret_cast<int*>(status), s);
    if (e == cudaSuccess) {
        k_from_chunked<<<sms * 8, 256, 0, s>>>(co, H, W, cout, static_cast<__nv_bfloat16*>(out));
        e = cudaGetLastError();
    }
    dev_free_async(ci, s);
    dev_free_async(co, s);
    dev_free_async(wpk, s);
    if (e != cudaSuccess) return cuda_fail(e, "conv3x3");
    return LFDPR_OK;
}

}  // extern "C"
