// Coarse-grid correction network: three periodic 3x3x3 convolutions
// (5 -> 32 -> 32 -> 5 channels, exact GELU after the first two) applied to a
// coarse solver state after each RK3 step, trained on the GPU.
//
// * Convolutions (forward, and the input gradient of the backward pass) are
//   implicit GEMMs on the tcgen05 tensor cores: M = 128 grid points per MMA,
//   N = the output channels of the three z taps of one (dy, dx) tap (they
//   share the A window), K = 9 (dy, dx) taps x input channels; BF16 operands
//   in shared memory as K-major core matrices, FP32 accumulators in TMEM.
// * A persistent, warp-specialised CTA per SM: one warp loads each tile's
//   input plus its periodic one-point halo with ONE TMA box into a two- or
//   three-stage ring, one thread issues the tile's MMAs from shifted
//   descriptors into one of two TMEM accumulator buffers, and eight
//   epilogue warps read the other buffer (bias, GELU or GELU', BF16 stores),
//   so loads, MMAs and epilogues of consecutive tiles overlap.  The weights
//   (B operand) stay in shared memory.  Activations are kept in a padded,
//   chunk-major layout whose one-point frame holds the periodic copies, so a
//   halo never wraps.  The input gradient is the same kernel with the
//   weights transposed in channels and flipped in taps.
// * The weight gradient sums over all grid points (K = points) on CUDA cores
//   in FP32, split over CTAs and reduced in a fixed order (deterministic).
// * MSE loss, Adam (FP32 master weights, BF16 copies in both GEMM layouts),
//   input normalisation, the residual update of the solver state, and the
//   centred box filter that makes training targets from fine-grid runs.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/gbfd.h"
#include "kernels.cuh"
#include "tcgen05.cuh"
#include "tiled_impl.cuh"

namespace gbfd {
bool ctx_view(gbfd_ctx *c, float **origin, Layout *L, int *nf, cudaStream_t *s);
}

namespace gbfd {
namespace cnn {

using bf16 = __nv_bfloat16;

constexpr int TAPS = 27;
constexpr int MT = 128;    // points per tile (MMA M)
constexpr int NC = 5;      // physical channels (lnrho, u_x, u_y, u_z, s)
constexpr int C0 = 16;     // padded input channels of layer 1
constexpr int CH = 32;     // hidden channels
constexpr int C3 = 16;     // padded output channels of layer 3

enum { EPI_GELU = 0, EPI_LINEAR = 1, EPI_DGELU = 2 };

// Packed FP32 parameters: W[co_pad][tap][ci_pad] then b[co_pad], per layer;
// padded channel counts per layer: (32, 16), (32, 32), (16, 32).
__host__ __device__ constexpr int dim_co(int l) { return l == 2 ? C3 : CH; }
__host__ __device__ constexpr int dim_ci(int l) { return l == 0 ? C0 : CH; }

__host__ __device__ constexpr int wcount(int l) { return dim_co(l) * TAPS * dim_ci(l); }
__host__ __device__ constexpr int pcount(int l) { return wcount(l) + dim_co(l); }
__host__ __device__ constexpr int poff(int l)
{
    return l == 0 ? 0 : (l == 1 ? pcount(0) : pcount(0) + pcount(1));
}
constexpr int kParams = pcount(0) + pcount(1) + pcount(2);
// real (unpadded) sizes, in the W[o][c][3][3][3] + b[o] order, layers 1..3
constexpr int kRealOut[3] = {CH, CH, NC};
constexpr int kRealIn[3] = {NC, CH, CH};
constexpr int kRealParams = (CH * NC * 27 + CH) + (CH * CH * 27 + CH) + (NC * CH * 27 + NC);

// element index of (row n, col k) of an N x K operand in core-matrix order
__host__ __device__ inline int core_idx(int n, int k, int K)
{
    return (n / 8) * (K * 8) + (k / 8) * 64 + (n % 8) * 8 + (k % 8);
}

__device__ __forceinline__ float gelu(float h) { return 0.5f * h * (1.0f + erff(h * 0.70710678118654752f)); }

__device__ __forceinline__ float gelu_grad(float h)
{
    return 0.5f * (1.0f + erff(h * 0.70710678118654752f)) +
           h * expf(-0.5f * h * h) * 0.39894228040143268f;
}

// Activations live in a padded, chunk-major layout: act[c8][b][zp][yp][xp][8]
// (BF16; c8 = channel / 8, padded coordinates xp = x + 1 in 0..n+1, the
// outermost ones holding the periodic copies of the opposite faces), so that
// a tile's one-point halo is one rectangular, in-bounds box and the 8
// channels of one chunk of one point are 16 contiguous bytes.  Whoever writes
// a point also writes its periodic copies.  Index below in units of 16-byte
// chunks.
__host__ __device__ __forceinline__ long long aidx(int c8, int b, int zp, int yp, int xp, int n,
                                                   int B)
{
    const long long m = n + 2;
    return ((((long long)c8 * B + b) * m + zp) * m + yp) * m + xp;
}

// Calls f(xp, yp, zp) for the padded position of interior point (x, y, z)
// and for each of its periodic copies in the one-point frame (up to 8 at a
// corner; n >= 2).
template <class F>
__device__ __forceinline__ void each_copy(int x, int y, int z, int n, F &&f)
{
    const int xs[2] = {x + 1, x == 0 ? n + 1 : 0}, nxs = (x == 0 || x == n - 1) ? 2 : 1;
    const int ys[2] = {y + 1, y == 0 ? n + 1 : 0}, nys = (y == 0 || y == n - 1) ? 2 : 1;
    const int zs[2] = {z + 1, z == 0 ? n + 1 : 0}, nzs = (z == 0 || z == n - 1) ? 2 : 1;
    for (int iz = 0; iz < nzs; ++iz)
        for (int iy = 0; iy < nys; ++iy)
            for (int ix = 0; ix < nxs; ++ix)
                f(xs[ix], ys[iy], zs[iz]);
}

struct ConvArgs {
    const bf16 *wB;      // [N][27*CIN] in core-matrix order
    const float *bias;   // [N]                      (EPI_GELU, EPI_LINEAR)
    float *hsave;        // [npts][N] pre-activation (EPI_GELU; NULL: not kept)
    bf16 *yb;            // padded chunk-major output (EPI_GELU: GELU(h), EPI_DGELU: dh)
    float *yf;           // [npts][8]                (EPI_LINEAR)
    const float *hprev;  // [npts][N]                (EPI_DGELU)
    int n;               // grid side
    int npts;            // batch * n^3
    int B;               // samples allocated in the padded arrays
    int *dev_error;
};

// A conv tile is TXT x TYT points in each of ZB consecutive z planes: one
// M = 128 MMA row block per plane, row r = point (x0 + r % TXT, y0 + r / TXT).
// Its input plus the one-point halo, HX x HY x HZ points of CIN channels, is
// ONE TMA box of the padded chunk-major input, (8 channels, HX, HY, HZ,
// CIN / 8 chunks): in shared memory chunk c of halo point (hx, hy, hz) sits at
// c * CS + ((hz * HY + hy) * HX + hx) * 16.  The A operand of halo plane hz
// and in-plane tap (dy, dx) is that buffer at a shifted start: core matrices
// of 8 x-consecutive rows (16-byte row stride), row groups one halo row apart
// (SBO = HX * 16), K chunks CS apart (LBO).
//
// The three z taps of one (dy, dx) read the same A window (halo plane hz
// feeds output planes hz - dz for dz = 0, 1, 2), so they are ONE MMA with
// their weights stacked along N (N = 3 NO for NO output channels): a
// tcgen05 MMA of M = 128, K = 16 costs about the same for N = 16 or 32 as for
// 96 (measured on GB300: 45 cycles for N <= 32, 56 for N = 96, 64 for 128),
// so merging the z taps cuts the MMA time per output plane by about 2.4 at
// ZB = 4.  Column group dz of the MMA of halo plane hz lands on output plane
// zo = hz - dz; placing plane zo's accumulator at column NO (ZB + 1 - zo)
// makes the three groups of every MMA consecutive columns at
// NO (ZB + 1 - hz).  Planes -2, -1, ZB and ZB + 1 catch the groups that fall
// outside the tile (never read).  Every MMA accumulates, so the buffers
// start at zero and the epilogue zeroes the columns it has read before
// handing the buffer back.
constexpr int TXT = 8, TYT = 16, ZB = 4;
constexpr int HX = TXT + 2, HY = TYT + 2, HZ = ZB + 2, HPTS = HX * HY * HZ;
static_assert(TXT * TYT == MT, "one MMA row block per tile plane");
constexpr int TAPS_XY = 9;  // (dy, dx) taps; dz is stacked along N

// Warp roles of the convolution CTA (one per SM, persistent over tiles):
// warp 0 issues the TMA halo loads, warp 1 the MMAs (and owns the TMEM
// allocation), warps 2-9 are the epilogue (warp w reads TMEM lanes
// 32 (w % 4) .. 32 (w % 4) + 31; warps 2-5 the first half of the output
// channels, 6-9 the second).
constexpr int CONV_THREADS = 320;
constexpr int EPI_WARPS = 8;
constexpr int NACC = 2;  // TMEM accumulator buffers

template <int CIN, int NO, int EPI>
struct ConvSmem {
    static constexpr int N = 3 * NO;          // MMA N: the three z taps' output channels
    static constexpr int K = TAPS_XY * CIN;   // B operand K: (dy, dx) taps x input channels
    static constexpr int CH8 = CIN / 8;
    static constexpr int B_BYTES = N * K * 2;
    static constexpr int CS = HPTS * 16;  // chunk stride of the TMA box
    static constexpr int A_BYTES = CH8 * CS;
    static constexpr int NSTAGE = CIN >= 32 ? 2 : 3;  // halo buffers
    static constexpr int A_OFF = (B_BYTES + 1023) / 1024 * 1024;
    static constexpr int A_PITCH = (A_BYTES + 1023) / 1024 * 1024;
    static constexpr int BAR_OFF = A_OFF + NSTAGE * A_PITCH;
    // full[NSTAGE], empty[NSTAGE], acc_full[NACC], acc_empty[NACC], then the
    // TMEM address, the abort flag and four issue / consume counts
    static constexpr int BYTES = BAR_OFF + (2 * NSTAGE + 2 * NACC) * 8 + 8 + 16;
    static constexpr int ACC_COLS = (ZB + 4) * NO;  // one accumulator buffer
    static constexpr int TCOLS = NACC * ACC_COLS <= 128 ? 128 : (NACC * ACC_COLS <= 256 ? 256 : 512);
    static_assert(NACC * ACC_COLS <= 512, "TMEM columns");
    static_assert(CS % 16 == 0 && (CS >> 4) < (1 << 14) && ((K * 16) >> 4) < (1 << 14),
                  "descriptor offsets");
    static_assert(BYTES <= 227 * 1024, "shared memory");
};

// Zeroes 16 (or 8) consecutive FP32 columns of this warp's 32 TMEM lanes and
// waits for the stores to complete.
__device__ __forceinline__ void tmem_zero16(uint32_t taddr)
{
    const uint32_t z = 0;
    __syncwarp();
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
        "{%1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1};\n\t"
        "tcgen05.wait::st.sync.aligned;" ::"r"(taddr),
        "r"(z)
        : "memory");
}

__device__ __forceinline__ void tmem_zero8(uint32_t taddr)
{
    const uint32_t z = 0;
    __syncwarp();
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %1, %1, %1, %1, %1, %1, %1};\n\t"
        "tcgen05.wait::st.sync.aligned;" ::"r"(taddr),
        "r"(z)
        : "memory");
}

// Programmatic dependent launch (a kernel launched with programmatic stream
// serialisation may start while its predecessor in the stream finishes):
// pdl_wait blocks until the predecessor grid has completed and its memory
// is visible; pdl_trigger lets this grid's dependant start once every CTA
// of this grid has triggered or exited.  Both are no-ops for a kernel
// launched without the attribute.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger()
{
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tiled::smem_u32(bar))
                 : "memory");
}

// Bounded wait that also gives up when another role has raised the CTA's
// abort flag; a wait that runs out (about 2 s) raises it.
__device__ __forceinline__ bool wait_or_abort(uint64_t *bar, uint32_t parity, volatile int *abort)
{
    if (tiled::mbar_try_wait(bar, parity))
        return true;
    const uint64_t t0 = tiled::global_ns();
    while (true) {
        if (tiled::mbar_try_wait(bar, parity))
            return true;
        if (*abort)
            return false;
        if (tiled::global_ns() - t0 > 2000000000ull) {
            *abort = 1;
            return false;
        }
    }
}

__device__ __forceinline__ void tile_origin(int tile, int n, int &x0, int &y0, int &z0, int &b)
{
    const int tx_n = (n + TXT - 1) / TXT, ty_n = (n + TYT - 1) / TYT, tz_n = (n + ZB - 1) / ZB;
    int r = tile;
    x0 = (r % tx_n) * TXT;
    r /= tx_n;
    y0 = (r % ty_n) * TYT;
    r /= ty_n;
    z0 = (r % tz_n) * ZB;
    b = r / tz_n;
}

template <int CIN, int NO, int EPI>
__global__ void __launch_bounds__(CONV_THREADS, 1)
    k_conv_tc(const __grid_constant__ CUtensorMap xmap, const ConvArgs a)
{
    using SM = ConvSmem<CIN, NO, EPI>;
    constexpr int NSTAGE = SM::NSTAGE;
    constexpr int KSTEPS = CIN / 16;  // MMAs per (dy, dx) tap and halo plane
    constexpr int SBO_B = SM::K * 16;
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char *sB = smem;
    unsigned char *sA = smem + SM::A_OFF;
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + SM::BAR_OFF);
    uint64_t *empty = full + NSTAGE;
    uint64_t *accf = empty + NSTAGE;
    uint64_t *acce = accf + NACC;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(acce + NACC);
    volatile int *abort = reinterpret_cast<volatile int *>(tslot + 1);
    int *cnt = reinterpret_cast<int *>(tslot + 2);  // issued, consumed, committed, drained
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;

    // epilogue geometry: two warps per TMEM lane quarter, each taking half
    // of the output channels
    constexpr int NH = NO / 2;  // channels per epilogue warp
    static_assert(NH == 16 || NH == 8, "epilogue column chunks");
    const int e = warp - 2;
    const int q = warp % 4, c0 = (e / 4) * NH;
    auto zero_cols = [&](uint32_t taddr) {
        if constexpr (NH == 16)
            tmem_zero16(taddr);
        else
            tmem_zero8(taddr);
    };

    // the weights (B operand) stay in shared memory for the whole launch
    for (int i = threadIdx.x; i < SM::B_BYTES / 16; i += CONV_THREADS)
        reinterpret_cast<uint4 *>(sB)[i] = reinterpret_cast<const uint4 *>(a.wB)[i];
    if (threadIdx.x == 0) {
        for (int s = 0; s < NSTAGE; ++s) {
            tiled::mbar_init(&full[s], 1);
            tiled::mbar_init(&empty[s], 1);
        }
        for (int s = 0; s < NACC; ++s) {
            tiled::mbar_init(&accf[s], 1);
            tiled::mbar_init(&acce[s], EPI_WARPS);  // one arrival per epilogue warp
        }
        *abort = 0;
        cnt[0] = cnt[1] = cnt[2] = cnt[3] = 0;
        tiled::fence_mbar_init();
    }
    if (warp == 1)
        tc::tmem_alloc(tslot, SM::TCOLS);
    tc::fence_smem_to_async();  // the weights, written by the generic proxy, feed the MMAs
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *reinterpret_cast<volatile uint32_t *>(tslot);
    // every MMA accumulates: both accumulator buffers start at zero
    if (warp >= 2) {
        const uint32_t tl = tmem + ((uint32_t)(q * 32) << 16) + c0;
#pragma unroll 1
        for (int j = 0; j < NACC * (ZB + 4); ++j)
            zero_cols(tl + j * NO);
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    // everything above (weights, barriers, TMEM) may overlap the tail of the
    // kernel before this one in the stream, which never writes the weights
    // (the input staging kernel, another convolution or the gradient
    // reduction); the activations it writes are read only below
    pdl_wait();
    pdl_trigger();
    const int n = a.n;
    const long long n3 = (long long)n * n * n;
    const int nb = (int)(a.npts / n3);
    const int ntiles = nb * ((n + ZB - 1) / ZB) * ((n + TYT - 1) / TYT) * ((n + TXT - 1) / TXT);

    if (warp == 0) {
        // producer: one halo box per tile into the stage the MMAs freed
        if (lane == 0) {
            int i = 0;
            for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++i) {
                const int s = i % NSTAGE;
                if (!wait_or_abort(&empty[s], ((i / NSTAGE) & 1) ^ 1, abort))
                    break;
                int x0, y0, z0, b;
                tile_origin(tile, n, x0, y0, z0, b);
                tiled::mbar_expect_tx(&full[s], SM::A_BYTES);
                // padded coordinates of the halo's first point: (x0 - 1) + 1;
                // x and the 8 channels of a chunk form one 160-byte row
                tiled::tma_load_4d(sA + s * SM::A_PITCH, &xmap, &full[s], 8 * x0, y0,
                                   b * (n + 2) + z0, 0);
                cnt[0] = i + 1;
            }
        }
    } else if (warp == 1) {
        // MMA issuer: per halo plane, 9 (dy, dx) taps x KSTEPS MMAs of
        // N = 3 NO into one of two accumulator buffers; the commits free the
        // halo stage and hand the accumulators to the epilogue
        if (lane == 0) {
            constexpr uint32_t idesc = tc::idesc_bf16_f32(MT, SM::N);
            // descriptors of the stage and weight bases; every tap's operand
            // is a compile-time byte offset from them (the start address is
            // the descriptor's low field, in 16-byte units, and shared
            // memory addresses stay below 2^18 bytes, so adding the offset
            // cannot carry into the next field)
            const uint64_t bd0 = tc::smem_desc(tc::smem_u32(sB), 128, SBO_B);
            const uint64_t ad0 = tc::smem_desc(tc::smem_u32(sA), SM::CS, HX * 16);
            int i = 0;
            for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++i) {
                const int s = i % NSTAGE, acc = i % NACC;
                if (!wait_or_abort(&full[s], (i / NSTAGE) & 1, abort))
                    break;
                cnt[1] = i + 1;
                if (!wait_or_abort(&acce[acc], ((i / NACC) & 1) ^ 1, abort))
                    break;
                tc::fence_after_sync();
                const uint64_t adst = ad0 + (uint64_t)((s * SM::A_PITCH) >> 4);
                const uint32_t dbuf = tmem + acc * SM::ACC_COLS;
#pragma unroll
                for (int hz = 0; hz < HZ; ++hz)
#pragma unroll
                    for (int t = 0; t < TAPS_XY; ++t) {
                        const int dy = t / 3, dx = t % 3;  // offset + 1
#pragma unroll
                        for (int k = 0; k < KSTEPS; ++k) {
                            const int aoff =
                                (((hz * HY + dy) * HX + dx) * 16 + 2 * k * SM::CS) >> 4;
                            tc::mma_bf16(dbuf + (uint32_t)(NO * (ZB + 1 - hz)),
                                         adst + (uint64_t)aoff,
                                         bd0 + (uint64_t)((t * KSTEPS + k) * 16), idesc, 1u);
                        }
                    }
                tc::commit(&empty[s]);
                tc::commit(&accf[acc]);
                cnt[2] = i + 1;
            }
        }
    } else {
        // epilogue, per tile plane: TMEM -> registers, zero those columns,
        // then bias / GELU / GELU' and the stores (with the periodic copies)
        const int r = q * 32 + lane;  // row of the M block = TMEM lane
        const int lx = r % TXT, ly = r / TXT;
        const uint32_t tl = tmem + ((uint32_t)(q * 32) << 16) + c0;
        float bias[NH];
#pragma unroll
        for (int j = 0; j < NH; ++j)
            bias[j] = (EPI == EPI_DGELU || c0 + j >= NO) ? 0.f : __ldg(a.bias + c0 + j);
        int i = 0;
        for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++i) {
            const int acc = i % NACC;
            // one lane waits, the warp follows it (the TMEM accesses below
            // are warp-collective)
            int ok = 0;
            if (lane == 0)
                ok = wait_or_abort(&accf[acc], (i / NACC) & 1, abort);
            if (!__shfl_sync(0xffffffffu, ok, 0))
                break;
            // the other lanes observe the completed phase too (it cannot
            // move on before this warp releases the buffer)
            if (lane != 0)
                (void)tiled::mbar_try_wait(&accf[acc], (i / NACC) & 1);
            tc::fence_after_sync();
            const uint32_t tb = tl + acc * SM::ACC_COLS;
            int x0, y0, z0, b;
            tile_origin(tile, n, x0, y0, z0, b);
            const int x = x0 + lx, y = y0 + ly;
#pragma unroll 1
            for (int zo = 0; zo < ZB; ++zo) {
                const uint32_t tp = tb + (uint32_t)(NO * (ZB + 1 - zo));
                float v[NH];
                if constexpr (NH == 16)
                    tc::tmem_ld16(tp, v);
                else
                    tc::tmem_ld8(tp, v);
                zero_cols(tp);
                const int z = z0 + zo;
                if (x >= n || y >= n || z >= n)
                    continue;
                const long long p = (long long)b * n3 + ((long long)z * n + y) * n + x;
                if constexpr (EPI == EPI_LINEAR) {
                    // five real output channels, all in the first half
                    if (c0 == 0) {
                        float4 *yo = reinterpret_cast<float4 *>(a.yf + p * 8);
                        yo[0] = make_float4(v[0] + bias[0], v[1] + bias[1], v[2] + bias[2],
                                            v[3] + bias[3]);
                        yo[1] = make_float4(v[4] + bias[4], 0.f, 0.f, 0.f);
                    }
                } else {
                    uint4 out[NH / 8];
#pragma unroll
                    for (int c = 0; c < NH; c += 8) {
                        float h[8];
                        if constexpr (EPI == EPI_GELU) {
#pragma unroll
                            for (int j = 0; j < 8; ++j)
                                h[j] = v[c + j] + bias[c + j];
                            if (a.hsave) {
                                float4 *hs = reinterpret_cast<float4 *>(a.hsave + p * NO + c0 + c);
                                hs[0] = make_float4(h[0], h[1], h[2], h[3]);
                                hs[1] = make_float4(h[4], h[5], h[6], h[7]);
                            }
#pragma unroll
                            for (int j = 0; j < 8; ++j)
                                h[j] = gelu(h[j]);
                        } else {
                            const float4 *hp =
                                reinterpret_cast<const float4 *>(a.hprev + p * NO + c0 + c);
                            const float4 h0 = __ldg(hp), h1 = __ldg(hp + 1);
                            const float hv[8] = {h0.x, h0.y, h0.z, h0.w, h1.x, h1.y, h1.z, h1.w};
#pragma unroll
                            for (int j = 0; j < 8; ++j)
                                h[j] = v[c + j] * gelu_grad(hv[j]);
                        }
                        __nv_bfloat162 o[4];
#pragma unroll
                        for (int j = 0; j < 4; ++j)
                            o[j] = __floats2bfloat162_rn(h[2 * j], h[2 * j + 1]);
                        out[c / 8] = *reinterpret_cast<uint4 *>(o);
                    }
                    uint4 *yb = reinterpret_cast<uint4 *>(a.yb);
                    each_copy(x, y, z, n, [&](int xp, int yp, int zp) {
#pragma unroll
                        for (int k8 = 0; k8 < NH / 8; ++k8)
                            yb[aidx(c0 / 8 + k8, b, zp, yp, xp, n, a.B)] = out[k8];
                    });
                }
            }
            // (the spill planes -2, -1, ZB, ZB + 1 keep accumulating: they are
            // never read, and their columns are no other plane's)
            tc::fence_before_sync();
            __syncwarp();
            if (lane == 0)
                mbar_arrive(&acce[acc]);
            if (e == 0 && lane == 0)
                cnt[3] = i + 1;
        }
    }
    __syncthreads();
    if (*abort) {
        // a wait gave up: let the copies and MMAs still in flight land
        // before the shared memory and TMEM go away (bounded, abort ignored)
        if (threadIdx.x == 0) {
            atomicExch(a.dev_error, 2);
            volatile int never = 0;
            for (int j = cnt[1]; j < cnt[0]; ++j)
                (void)wait_or_abort(&full[j % NSTAGE], (j / NSTAGE) & 1, &never);
            for (int j = cnt[3]; j < cnt[2]; ++j)
                (void)wait_or_abort(&accf[j % NACC], (j / NACC) & 1, &never);
        }
        __syncthreads();
    }
    tc::fence_after_sync();
    if (warp == 1)
        tc::tmem_dealloc(tmem, SM::TCOLS);
}

// Weight (and bias) gradient of one layer, summed over this CTA's share of
// the points: dW[co][tap][ci] += dY[p][co] X[p + tap][ci]; db[co] += dY[p][co].
// dY and X are padded chunk-major activations (B samples allocated), so the
// neighbour p + tap is read without any wrap arithmetic.
template <int CO, int CI>
__global__ void __launch_bounds__(TAPS *(CI / 4)) k_wgrad(const bf16 *__restrict__ dY,
                                                          const bf16 *__restrict__ X, int n,
                                                          int npts, int B, float *__restrict__ part)
{
    constexpr int NT = TAPS * (CI / 4);
    __shared__ __align__(16) bf16 sdy[MT * CO];
    const int t = threadIdx.x;
    const int tap = t / (CI / 4), cq = t % (CI / 4);
    const int dz = tap / 9 - 1, dyo = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
    const int n2 = n * n, n3 = n2 * n;
    float acc[CO][4];
    float db[CO];
#pragma unroll
    for (int c = 0; c < CO; ++c) {
        db[c] = 0.f;
#pragma unroll
        for (int i = 0; i < 4; ++i)
            acc[c][i] = 0.f;
    }
    const long long chunk = ((long long)npts + gridDim.x - 1) / gridDim.x;
    const long long p0 = chunk * blockIdx.x;
    const long long p1 = min((long long)npts, p0 + chunk);
    const uint4 *dY4 = reinterpret_cast<const uint4 *>(dY);
    for (long long base = p0; base < p1; base += MT) {
        const int cnt = (int)min((long long)MT, p1 - base);
        __syncthreads();
        for (int i = t; i < cnt * (CO / 8); i += NT) {
            const int j = i / (CO / 8), c8 = i % (CO / 8);
            const long long p = base + j;
            const int b = (int)(p / n3);
            int r = (int)(p - (long long)b * n3);
            const int z = r / n2;
            r -= z * n2;
            reinterpret_cast<uint4 *>(sdy)[i] =
                __ldg(dY4 + aidx(c8, b, z + 1, r / n + 1, r % n + 1, n, B));
        }
        __syncthreads();
        for (int j = 0; j < cnt; ++j) {
            const long long p = base + j;
            const int b = (int)(p / n3);
            int r = (int)(p - (long long)b * n3);
            const int z = r / n2;
            r -= z * n2;
            const int y = r / n;
            const int x = r - y * n;
            const long long q =
                aidx(cq / 2, b, z + 1 + dz, y + 1 + dyo, x + 1 + dx, n, B) * 8 + (cq % 2) * 4;
            const uint2 xr = __ldg(reinterpret_cast<const uint2 *>(X + q));
            const float2 x01 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&xr.x));
            const float2 x23 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&xr.y));
            const float xv[4] = {x01.x, x01.y, x23.x, x23.y};
#pragma unroll
            for (int c = 0; c < CO; c += 2) {
                const float2 d = __bfloat1622float2(
                    *reinterpret_cast<const __nv_bfloat162 *>(sdy + j * CO + c));
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    acc[c][i] += d.x * xv[i];
                    acc[c + 1][i] += d.y * xv[i];
                }
                db[c] += d.x;
                db[c + 1] += d.y;
            }
        }
    }
    float *out = part + (long long)blockIdx.x * (CO * TAPS * CI + CO);
#pragma unroll
    for (int c = 0; c < CO; ++c)
#pragma unroll
        for (int i = 0; i < 4; ++i)
            out[(c * TAPS + tap) * CI + 4 * cq + i] = acc[c][i];
    if (t == 0)
#pragma unroll
        for (int c = 0; c < CO; ++c)
            out[CO * TAPS * CI + c] = db[c];
}

// g[i] = sum over CTAs of part[cta][i], fixed order.
__global__ void k_reduce_parts(const float *__restrict__ part, int nparts, int count,
                               float *__restrict__ g)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count)
        return;
    float s = 0.f;
    for (int c = 0; c < nparts; ++c)
        s += part[(long long)c * count + i];
    g[i] = s;
}

// Normalised BF16 input of layer 1 (C0 = 16 channels, zero beyond the nf
// physical fields) at point (b, x, y, z) into the padded chunk-major x0,
// with its periodic copies.
__device__ __forceinline__ void put_input(bf16 *x0, const float *v, int b, int x, int y, int z,
                                          int n, int B)
{
    __nv_bfloat162 o[8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
        o[i] = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
    const uint4 c0 = reinterpret_cast<uint4 *>(o)[0], c1 = reinterpret_cast<uint4 *>(o)[1];
    uint4 *dst = reinterpret_cast<uint4 *>(x0);
    each_copy(x, y, z, n, [&](int xp, int yp, int zp) {
        dst[aidx(0, b, zp, yp, xp, n, B)] = c0;
        dst[aidx(1, b, zp, yp, xp, n, B)] = c1;
    });
}

// Layer-1 input from compact FP32 states [batch][5][n^3] (nf fields present).
__global__ void k_input_compact(const float *__restrict__ xs, int nf, int n, int npts, int B,
                                const float *__restrict__ mean, const float *__restrict__ stdv,
                                bf16 *__restrict__ x0)
{
    pdl_trigger();  // the first convolution may start its prologue
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npts)
        return;
    const int n3 = n * n * n;
    const int b = p / n3, r = p - b * n3;
    float v[C0];
#pragma unroll
    for (int c = 0; c < C0; ++c)
        v[c] = (c < nf) ? (xs[((long long)b * NC + c) * n3 + r] - mean[c]) / stdv[c] : 0.f;
    put_input(x0, v, b, r % n, (r / n) % n, r / (n * n), n, B);
}

// Same from a solver context's padded FP32 state (one box, batch 1).
__global__ void k_input_state(const float *__restrict__ st, Layout L, int nf, int B,
                              const float *__restrict__ mean, const float *__restrict__ stdv,
                              bf16 *__restrict__ x0)
{
    pdl_trigger();  // the first convolution may start its prologue
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = L.nx;
    if (p >= n * n * n)
        return;
    const int z = p / (n * n), y = (p / n) % n, x = p % n;
    float v[C0];
#pragma unroll
    for (int c = 0; c < C0; ++c)
        v[c] = (c < nf) ? (st[lidx(L, c, z, y, x)] - mean[c]) / stdv[c] : 0.f;
    put_input(x0, v, 0, x, y, z, n, B);
}

// state += std_out * y (the de-normalised predicted residual), ghosts kept.
__global__ void k_apply(float *__restrict__ st, Layout L, int nf, const float *__restrict__ y,
                        const float *__restrict__ sout)
{
    pdl_wait();  // launched to overlap the last convolution's tail
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = L.nx;
    if (p >= n * n * n)
        return;
    const int z = p / (n * n), yy = (p / n) % n, x = p % n;
    for (int f = 0; f < nf; ++f) {
        const float v = st[lidx(L, f, z, yy, x)] + sout[f] * y[(long long)p * 8 + f];
        store_ghosted(st, L, f, z, yy, x, v);
    }
}

// Normalised output [batch][5][n^3] from the layer-3 rows (tests, inference).
__global__ void k_output_compact(const float *__restrict__ y, int n3, int npts,
                                 float *__restrict__ out)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npts)
        return;
    const int b = p / n3, r = p - b * n3;
    for (int c = 0; c < NC; ++c)
        out[((long long)b * NC + c) * n3 + r] = y[(long long)p * 8 + c];
}

// MSE of the normalised residual: t = (target - x) / std_out; loss partial
// sums per block (FP64) and dY3 = 2 (y - t) / count in BF16, channels-last.
__global__ void k_loss(const float *__restrict__ y, const float *__restrict__ xs,
                       const float *__restrict__ ts, const float *__restrict__ sout, int nf,
                       int n, int npts, int B, float inv_count, bf16 *__restrict__ dy3,
                       double *__restrict__ part)
{
    const int n3 = n * n * n;
    __shared__ double sh[256];
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    double l = 0.0;
    if (p < npts) {
        const int b = p / n3, r = p - b * n3;
        float d[C3];
#pragma unroll
        for (int c = 0; c < C3; ++c)
            d[c] = 0.f;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const long long i = ((long long)b * NC + c) * n3 + r;
            const float t = c < nf ? (ts[i] - xs[i]) / sout[c] : 0.f;
            const float e = y[(long long)p * 8 + c] - t;
            l += (double)e * (double)e;
            d[c] = 2.f * e * inv_count;
        }
        // dY3 into the padded chunk-major layout, with its periodic copies
        put_input(dy3, d, b, r % n, (r / n) % n, r / (n * n), n, B);
    }
    sh[threadIdx.x] = l;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        part[blockIdx.x] = sh[0];
}

__global__ void k_sum_double(const double *__restrict__ part, int n, double *__restrict__ out)
{
    __shared__ double sh[256];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += 256)
        s += part[i];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int k = 128; k > 0; k >>= 1) {
        if (threadIdx.x < k)
            sh[threadIdx.x] += sh[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        *out = sh[0];
}

struct PackArgs {
    float *w, *m, *v;  // FP32 master parameters and Adam moments [kParams]
    const float *g;    // gradients [kParams] (NULL: pack only)
    float lr, b1, b2, eps, bc1, bc2;
    bf16 *fwd[3];      // forward B operands, layer l: [dz][co][9*ci]
    bf16 *bwd[3];      // input-gradient B operands (layers 2, 3): [dz][ci][9*co]
    float *bias[3];    // FP32 biases [co]
};

// Adam step (Kingma & Ba 2015) on the master weights, then the BF16 GEMM
// copies, tap = (dz, dy, dx) = 9 dz + t: forward B[dz CO + co][t CI + ci];
// input-gradient B'[dz' CI + ci][t' CO + co] for the flipped tap
// (dz', t') of 26 - tap (channels transposed).
__global__ void k_adam_pack(PackArgs a)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kParams)
        return;
    float w = a.w[i];
    if (a.g) {
        const float g = a.g[i];
        const float m = a.b1 * a.m[i] + (1.f - a.b1) * g;
        const float v = a.b2 * a.v[i] + (1.f - a.b2) * g * g;
        a.m[i] = m;
        a.v[i] = v;
        w -= a.lr * (m / a.bc1) / (sqrtf(v / a.bc2) + a.eps);
        a.w[i] = w;
    }
    int l = i < poff(1) ? 0 : (i < poff(2) ? 1 : 2);
    const int j = i - poff(l);
    const int CO = dim_co(l), CI = dim_ci(l);
    if (j >= wcount(l)) {
        a.bias[l][j - wcount(l)] = w;
        return;
    }
    const int co = j / (TAPS * CI), tap = (j / CI) % TAPS, ci = j % CI;
    // rows: the three z taps' output channels stacked (dz * CO + co); K:
    // the (dy, dx) tap, then the input channel
    a.fwd[l][core_idx((tap / 9) * CO + co, (tap % 9) * CI + ci, TAPS_XY * CI)] =
        __float2bfloat16_rn(w);
    if (l > 0) {
        const int tf = TAPS - 1 - tap;  // flipped tap
        a.bwd[l][core_idx((tf / 9) * CI + ci, (tf % 9) * CO + co, TAPS_XY * CO)] =
            __float2bfloat16_rn(w);
    }
}

// Centred box filter: coarse vertex I sits on fine vertex r I; per axis the
// weights are (1/2, 1, ..., 1, 1/2) / r over fine offsets -r/2..r/2.
__global__ void k_box_filter(const float *__restrict__ fine, Layout L, int nf, int r,
                             float *__restrict__ out)
{
    const int nc = L.nx / r;
    const long long nc3 = (long long)nc * nc * nc;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nc3 * nf)
        return;
    const int f = (int)(i / nc3);
    const long long q = i - f * nc3;
    const int Z = (int)(q / ((long long)nc * nc)), Y = (int)((q / nc) % nc), X = (int)(q % nc);
    const int h = r / 2;
    double acc = 0.0;
    for (int a = -h; a <= h; ++a) {
        const double wa = (a == -h || a == h) ? 0.5 : 1.0;
        const int z = ((r * Z + a) % L.nz + L.nz) % L.nz;
        for (int b = -h; b <= h; ++b) {
            const double wb = (b == -h || b == h) ? 0.5 : 1.0;
            const int y = ((r * Y + b) % L.ny + L.ny) % L.ny;
            for (int c = -h; c <= h; ++c) {
                const double wc = (c == -h || c == h) ? 0.5 : 1.0;
                const int x = ((r * X + c) % L.nx + L.nx) % L.nx;
                acc += wa * wb * wc * (double)fine[lidx(L, f, z, y, x)];
            }
        }
    }
    out[i] = (float)(acc / ((double)r * r * r));
}

}  // namespace cnn
}  // namespace gbfd

using namespace gbfd;
using namespace gbfd::cnn;

struct gbfd_cnn {
    int n, batch, npts_max;
    cudaStream_t stream;
    char *ws;
    size_t ws_bytes;
    float *w, *m, *v, *g;
    bf16 *fwd[3], *bwd[3];
    float *bias[3];
    float *norm;  // mean_in[5], std_in[5], std_out[5]
    bf16 *x0, *a1, *a2, *dy3, *dh2, *dh1;
    float *h1, *h2, *y3;
    float *parts;
    int nparts;
    double *lparts, *loss;
    int *derr;
    int adam_t;
    int grid_conv;      // CTAs per convolution launch (each walks its share of the tiles)
    int grid_default;   // one per SM
    // TMA maps of the convolution inputs (padded chunk-major activations)
    CUtensorMap map_x0, map_a1, map_a2, map_dy3, map_dh2;
    int64_t launches;
    char err[512];
};

namespace {

thread_local char g_cnn_err[512];

void cerr(gbfd_cnn *c, const char *fmt, ...)
{
    char *buf = c ? c->err : g_cnn_err;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, 512, fmt, ap);
    va_end(ap);
}

gbfd_status ccuda(gbfd_cnn *c, cudaError_t e, const char *what)
{
    cerr(c, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
    return GBFD_ERR_CUDA;
}

size_t al(size_t v) { return (v + 1023) & ~(size_t)1023; }

struct CnnPlan {
    size_t off[32];
    size_t total;
    int nparts;
};

constexpr int kWgradParts = 296;  // CTAs of the weight-gradient kernels

CnnPlan plan_for(int n, int batch)
{
    CnnPlan pl;
    const size_t np = (size_t)batch * n * n * n;
    const size_t npad = (size_t)batch * (n + 2) * (n + 2) * (n + 2);  // padded activations
    const size_t sizes[] = {
        kParams * 4, kParams * 4, kParams * 4, kParams * 4,  // w m v g
        (size_t)CH * TAPS * C0 * 2, (size_t)CH * TAPS * CH * 2, (size_t)C3 * TAPS * CH * 2,  // fwd
        (size_t)C0 * TAPS * CH * 2, (size_t)CH * TAPS * CH * 2, (size_t)CH * TAPS * C3 * 2,  // bwd
        CH * 4, CH * 4, C3 * 4, 64 * 4,                                   // biases, norm
        npad * C0 * 2, npad * CH * 2, npad * CH * 2, npad * C3 * 2, npad * CH * 2,
        npad * CH * 2,                                                    // bf16 acts
        np * CH * 4, np * CH * 4, np * 8 * 4,                             // h1 h2 y3
        (size_t)kWgradParts * (CH * TAPS * CH + CH) * 4,                 // parts
        ((np + 255) / 256 + 8) * 8, 64, 256};
    size_t off = 0;
    const int cnt = sizeof(sizes) / sizeof(sizes[0]);
    for (int i = 0; i < cnt; ++i) {
        pl.off[i] = off;
        off = al(off + sizes[i]);
    }
    pl.total = off;
    pl.nparts = kWgradParts;
    return pl;
}

template <int CIN, int N, int EPI>
cudaError_t conv(gbfd_cnn *c, const CUtensorMap &xmap, const ConvArgs &a)
{
    using SM = ConvSmem<CIN, N, EPI>;
    auto k = k_conv_tc<CIN, N, EPI>;
    // the shared-memory opt-in once per device (it is a per-device attribute
    // of the kernel; the call costs host time on every launch otherwise)
    static std::atomic<unsigned long long> opted{0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return e;
    const unsigned long long bit = 1ull << (dev & 63);
    if (dev >= 64 || !(opted.load() & bit)) {
        e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, SM::BYTES);
        if (e != cudaSuccess)
            return e;
        if (dev < 64)
            opted.fetch_or(bit);
    }
    const int n = a.n;
    const long long ntiles = (long long)(a.npts / ((long long)n * n * n)) * ((n + ZB - 1) / ZB) *
                             ((n + TYT - 1) / TYT) * ((n + TXT - 1) / TXT);
    // persistent: one CTA per SM walking the tiles (fewer on request),
    // launched so that its prologue overlaps the previous kernel's tail
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)std::min<long long>(ntiles, c->grid_conv));
    cfg.blockDim = dim3(CONV_THREADS);
    cfg.dynamicSmemBytes = SM::BYTES;
    cfg.stream = c->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, k, xmap, a);
    c->launches++;
    return e != cudaSuccess ? e : cudaGetLastError();
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

// TMA map of a padded chunk-major activation of cin channels (B samples on
// an n^3 grid): dims (8 (n + 2) values = x and the 8 channels of a chunk,
// n + 2, (n + 2) B, cin / 8), box = one conv tile's halo, (8 HX, HY, HZ,
// cin / 8): 160-byte rows.
bool encode_act_map(CUtensorMap *m, const bf16 *base, int n, int B, int cin)
{
    PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
    if (!fn)
        return false;
    const cuuint64_t np2 = (cuuint64_t)(n + 2);
    const cuuint64_t dims[4] = {8 * np2, np2, np2 * (cuuint64_t)B, (cuuint64_t)(cin / 8)};
    const cuuint64_t strides[3] = {np2 * 16, np2 * np2 * 16, np2 * np2 * np2 * B * 16};
    const cuuint32_t box[4] = {8 * HX, HY, HZ, (cuuint32_t)(cin / 8)};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<bf16 *>(base), dims, strides, box,
              estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

cudaError_t pack(gbfd_cnn *c, const float *g, float lr)
{
    PackArgs a;
    a.w = c->w;
    a.m = c->m;
    a.v = c->v;
    a.g = g;
    a.lr = lr;
    a.b1 = 0.9f;
    a.b2 = 0.999f;
    a.eps = 1e-8f;
    a.bc1 = 1.f - powf(0.9f, (float)c->adam_t);
    a.bc2 = 1.f - powf(0.999f, (float)c->adam_t);
    for (int l = 0; l < 3; ++l) {
        a.fwd[l] = c->fwd[l];
        a.bwd[l] = c->bwd[l];
        a.bias[l] = c->bias[l];
    }
    k_adam_pack<<<(kParams + 255) / 256, 256, 0, c->stream>>>(a);
    c->launches++;
    return cudaGetLastError();
}

// forward of `npts` points whose layer-1 input is already in x0; `keep`
// saves the pre-activations for the backward pass (training only)
cudaError_t forward(gbfd_cnn *c, int npts, bool keep)
{
    ConvArgs a;
    memset(&a, 0, sizeof a);
    a.n = c->n;
    a.npts = npts;
    a.B = c->batch;
    a.dev_error = c->derr;
    a.wB = c->fwd[0];
    a.bias = c->bias[0];
    a.hsave = keep ? c->h1 : nullptr;
    a.yb = c->a1;
    cudaError_t e = conv<C0, CH, EPI_GELU>(c, c->map_x0, a);
    if (e != cudaSuccess)
        return e;
    a.wB = c->fwd[1];
    a.bias = c->bias[1];
    a.hsave = keep ? c->h2 : nullptr;
    a.yb = c->a2;
    e = conv<CH, CH, EPI_GELU>(c, c->map_a1, a);
    if (e != cudaSuccess)
        return e;
    a.wB = c->fwd[2];
    a.bias = c->bias[2];
    a.hsave = nullptr;
    a.yb = nullptr;
    a.yf = c->y3;
    return conv<CH, C3, EPI_LINEAR>(c, c->map_a2, a);
}

template <int CO, int CI>
cudaError_t wgrad(gbfd_cnn *c, const bf16 *dY, const bf16 *X, int npts, float *g)
{
    k_wgrad<CO, CI><<<c->nparts, TAPS * (CI / 4), 0, c->stream>>>(dY, X, c->n, npts, c->batch,
                                                                    c->parts);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return e;
    const int count = CO * TAPS * CI + CO;
    k_reduce_parts<<<(count + 255) / 256, 256, 0, c->stream>>>(c->parts, c->nparts, count, g);
    c->launches += 2;
    return cudaGetLastError();
}

// loss, backward and gradients for `batch` samples (x0 and y3 from forward)
cudaError_t backward(gbfd_cnn *c, const float *xs, const float *ts, int nf, int batch)
{
    const int n3 = c->n * c->n * c->n, npts = batch * n3;
    const int blocks = (npts + 255) / 256;
    const float *sout = c->norm + 10;
    k_loss<<<blocks, 256, 0, c->stream>>>(c->y3, xs, ts, sout, nf, c->n, npts, c->batch,
                                          1.0f / ((float)NC * npts), c->dy3, c->lparts);
    k_sum_double<<<1, 256, 0, c->stream>>>(c->lparts, blocks, c->loss);
    c->launches += 2;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return e;
    // layer 3: weight gradient, then input gradient through GELU'(h2)
    e = wgrad<C3, CH>(c, c->dy3, c->a2, npts, c->g + poff(2));
    if (e != cudaSuccess)
        return e;
    ConvArgs a;
    memset(&a, 0, sizeof a);
    a.n = c->n;
    a.npts = npts;
    a.dev_error = c->derr;
    a.B = c->batch;
    a.wB = c->bwd[2];
    a.hprev = c->h2;
    a.yb = c->dh2;
    e = conv<C3, CH, EPI_DGELU>(c, c->map_dy3, a);
    if (e != cudaSuccess)
        return e;
    // layer 2
    e = wgrad<CH, CH>(c, c->dh2, c->a1, npts, c->g + poff(1));
    if (e != cudaSuccess)
        return e;
    a.wB = c->bwd[1];
    a.hprev = c->h1;
    a.yb = c->dh1;
    e = conv<CH, CH, EPI_DGELU>(c, c->map_dh2, a);
    if (e != cudaSuccess)
        return e;
    // layer 1: weight gradient only
    return wgrad<CH, C0>(c, c->dh1, c->x0, npts, c->g + poff(0));
}

gbfd_status check(gbfd_cnn *c, int batch)
{
    if (!c)
        return GBFD_ERR_INVALID_ARG;
    if (batch < 1 || batch > c->batch) {
        cerr(c, "batch %d outside 1..%d", batch, c->batch);
        return GBFD_ERR_INVALID_ARG;
    }
    return GBFD_OK;
}

}  // namespace

extern "C" {

size_t gbfd_cnn_workspace_bytes(int n, int batch)
{
    if (n < 4 || n > 512 || batch < 1 || (long long)batch * n * n * n > (1LL << 30))
        return 0;
    return plan_for(n, batch).total;
}

gbfd_status gbfd_cnn_init(int n, int batch, void *workspace, size_t workspace_bytes, void *stream,
                          gbfd_cnn **out)
{
    if (!out) {
        cerr(nullptr, "out is NULL");
        return GBFD_ERR_INVALID_ARG;
    }
    *out = nullptr;
    const size_t need = gbfd_cnn_workspace_bytes(n, batch);
    if (need == 0) {
        cerr(nullptr, "cnn: n must be in 4..512, batch >= 1, batch*n^3 <= 2^30");
        return GBFD_ERR_INVALID_ARG;
    }
    if (!workspace || ((uintptr_t)workspace & 1023) || workspace_bytes < need) {
        cerr(nullptr, "cnn: workspace must be 1024-byte aligned with >= %zu bytes", need);
        return GBFD_ERR_WORKSPACE;
    }
    gbfd_cnn *c = new (std::nothrow) gbfd_cnn();
    if (!c) {
        cerr(nullptr, "out of host memory");
        return GBFD_ERR_INVALID_ARG;
    }
    CnnPlan pl = plan_for(n, batch);
    c->n = n;
    c->batch = batch;
    c->npts_max = batch * n * n * n;
    c->stream = (cudaStream_t)stream;
    c->ws = (char *)workspace;
    c->ws_bytes = workspace_bytes;
    char *b = c->ws;
    int k = 0;
    c->w = (float *)(b + pl.off[k++]);
    c->m = (float *)(b + pl.off[k++]);
    c->v = (float *)(b + pl.off[k++]);
    c->g = (float *)(b + pl.off[k++]);
    for (int l = 0; l < 3; ++l)
        c->fwd[l] = (bf16 *)(b + pl.off[k++]);
    for (int l = 0; l < 3; ++l)
        c->bwd[l] = (bf16 *)(b + pl.off[k++]);
    for (int l = 0; l < 3; ++l)
        c->bias[l] = (float *)(b + pl.off[k++]);
    c->norm = (float *)(b + pl.off[k++]);
    c->x0 = (bf16 *)(b + pl.off[k++]);
    c->a1 = (bf16 *)(b + pl.off[k++]);
    c->a2 = (bf16 *)(b + pl.off[k++]);
    c->dy3 = (bf16 *)(b + pl.off[k++]);
    c->dh2 = (bf16 *)(b + pl.off[k++]);
    c->dh1 = (bf16 *)(b + pl.off[k++]);
    c->h1 = (float *)(b + pl.off[k++]);
    c->h2 = (float *)(b + pl.off[k++]);
    c->y3 = (float *)(b + pl.off[k++]);
    c->parts = (float *)(b + pl.off[k++]);
    c->lparts = (double *)(b + pl.off[k++]);
    c->loss = (double *)(b + pl.off[k++]);
    c->derr = (int *)(b + pl.off[k++]);
    c->nparts = pl.nparts;
    c->adam_t = 0;
    c->launches = 0;
    c->err[0] = 0;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    c->grid_conv = c->grid_default = sms > 0 ? sms : 1;
    if (e == cudaSuccess &&
        !(encode_act_map(&c->map_x0, c->x0, n, batch, C0) &&
          encode_act_map(&c->map_a1, c->a1, n, batch, CH) &&
          encode_act_map(&c->map_a2, c->a2, n, batch, CH) &&
          encode_act_map(&c->map_dy3, c->dy3, n, batch, C3) &&
          encode_act_map(&c->map_dh2, c->dh2, n, batch, CH))) {
        cerr(nullptr, "cnn init: TMA descriptor encoding failed");
        delete c;
        return GBFD_ERR_CUDA;
    }
    if (e == cudaSuccess)
        e = cudaMemsetAsync(c->ws, 0, pl.total, c->stream);
    // identity normalisation until set
    std::vector<float> nm(64, 0.f);
    for (int i = 0; i < 5; ++i)
        nm[5 + i] = nm[10 + i] = 1.f;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->norm, nm.data(), 64 * 4, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        ccuda(nullptr, e, "cnn init");
        delete c;
        return GBFD_ERR_CUDA;
    }
    *out = c;
    return GBFD_OK;
}

gbfd_status gbfd_cnn_destroy(gbfd_cnn *c)
{
    delete c;
    return GBFD_OK;
}

gbfd_status gbfd_cnn_set_option(gbfd_cnn *c, int key, int64_t value)
{
    if (!c)
        return GBFD_ERR_INVALID_ARG;
    switch (key) {
    case GBFD_CNN_OPT_CONV_GRID:
        if (value < 0 || value > (1 << 20))
            break;
        c->grid_conv = value == 0 ? c->grid_default : (int)value;
        return GBFD_OK;
    case GBFD_CNN_OPT_WGRAD_PARTS:
        if (value < 0 || value > kWgradParts)
            break;
        c->nparts = value == 0 ? kWgradParts : (int)value;
        return GBFD_OK;
    default:
        break;
    }
    cerr(c, "cnn set_option: bad key %d or value %lld", key, (long long)value);
    return GBFD_ERR_INVALID_ARG;
}

gbfd_status gbfd_cnn_set_params(gbfd_cnn *c, const float *params)
{
    if (!c || !params) {
        cerr(c, "cnn set_params: NULL argument");
        return GBFD_ERR_INVALID_ARG;
    }
    std::vector<float> packed(kParams, 0.f);
    const float *src = params;
    for (int l = 0; l < 3; ++l) {
        const int CO = dim_co(l), CI = dim_ci(l);
        for (int o = 0; o < kRealOut[l]; ++o)
            for (int ci = 0; ci < kRealIn[l]; ++ci)
                for (int t = 0; t < TAPS; ++t)
                    packed[poff(l) + (o * TAPS + t) * CI + ci] = src[(o * kRealIn[l] + ci) * TAPS + t];
        src += kRealOut[l] * kRealIn[l] * TAPS;
        for (int o = 0; o < kRealOut[l]; ++o)
            packed[poff(l) + CO * TAPS * CI + o] = src[o];
        src += kRealOut[l];
    }
    cudaError_t e =
        cudaMemcpyAsync(c->w, packed.data(), kParams * 4, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(c->m, 0, kParams * 4, c->stream);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(c->v, 0, kParams * 4, c->stream);
    c->adam_t = 0;
    if (e == cudaSuccess)
        e = pack(c, nullptr, 0.f);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(c->stream);
    return e == cudaSuccess ? GBFD_OK : ccuda(c, e, "cnn set_params");
}

// unpack a padded parameter vector (device) into the real-size host layout
static gbfd_status unpack(gbfd_cnn *c, const float *dev, float *host)
{
    std::vector<float> packed(kParams);
    cudaError_t e =
        cudaMemcpyAsync(packed.data(), dev, kParams * 4, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess)
        return ccuda(c, e, "cnn read parameters");
    float *dst = host;
    for (int l = 0; l < 3; ++l) {
        const int CO = dim_co(l), CI = dim_ci(l);
        for (int o = 0; o < kRealOut[l]; ++o)
            for (int ci = 0; ci < kRealIn[l]; ++ci)
                for (int t = 0; t < TAPS; ++t)
                    dst[(o * kRealIn[l] + ci) * TAPS + t] = packed[poff(l) + (o * TAPS + t) * CI + ci];
        dst += kRealOut[l] * kRealIn[l] * TAPS;
        for (int o = 0; o < kRealOut[l]; ++o)
            dst[o] = packed[poff(l) + CO * TAPS * CI + o];
        dst += kRealOut[l];
    }
    return GBFD_OK;
}

gbfd_status gbfd_cnn_get_params(gbfd_cnn *c, float *params)
{
    if (!c || !params) {
        cerr(c, "cnn get_params: NULL argument");
        return GBFD_ERR_INVALID_ARG;
    }
    return unpack(c, c->w, params);
}

int gbfd_cnn_param_count(void) { return kRealParams; }

gbfd_status gbfd_cnn_set_norm(gbfd_cnn *c, const float *mean_in, const float *std_in,
                              const float *std_out)
{
    if (!c || !mean_in || !std_in || !std_out) {
        cerr(c, "cnn set_norm: NULL argument");
        return GBFD_ERR_INVALID_ARG;
    }
    float nm[64] = {0};
    for (int i = 0; i < 5; ++i) {
        if (!(std_in[i] > 0) || !(std_out[i] > 0)) {
            cerr(c, "cnn set_norm: standard deviations must be > 0");
            return GBFD_ERR_INVALID_ARG;
        }
        nm[i] = mean_in[i];
        nm[5 + i] = std_in[i];
        nm[10 + i] = std_out[i];
    }
    cudaError_t e = cudaMemcpyAsync(c->norm, nm, sizeof nm, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(c->stream);
    return e == cudaSuccess ? GBFD_OK : ccuda(c, e, "cnn set_norm");
}

gbfd_status gbfd_cnn_forward(gbfd_cnn *c, const float *xs, int nf, int batch, float *ys)
{
    gbfd_status st = check(c, batch);
    if (st != GBFD_OK)
        return st;
    if (!xs || !ys || (nf != 4 && nf != 5)) {
        cerr(c, "cnn forward: bad arguments");
        return GBFD_ERR_INVALID_ARG;
    }
    const int n3 = c->n * c->n * c->n, npts = batch * n3;
    k_input_compact<<<(npts + 255) / 256, 256, 0, c->stream>>>(xs, nf, c->n, npts, c->batch,
                                                                c->norm, c->norm + 5, c->x0);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
        e = forward(c, npts, false);
    if (e == cudaSuccess) {
        k_output_compact<<<(npts + 255) / 256, 256, 0, c->stream>>>(c->y3, n3, npts, ys);
        e = cudaGetLastError();
    }
    c->launches += 2;
    return e == cudaSuccess ? GBFD_OK : ccuda(c, e, "cnn forward");
}

gbfd_status gbfd_cnn_gradients(gbfd_cnn *c, const float *xs, const float *ts, int nf, int batch,
                               float *grads, double *loss)
{
    gbfd_status st = check(c, batch);
    if (st != GBFD_OK)
        return st;
    if (!xs || !ts || (nf != 4 && nf != 5)) {
        cerr(c, "cnn gradients: bad arguments");
        return GBFD_ERR_INVALID_ARG;
    }
    const int n3 = c->n * c->n * c->n, npts = batch * n3;
    k_input_compact<<<(npts + 255) / 256, 256, 0, c->stream>>>(xs, nf, c->n, npts, c->batch,
                                                                c->norm, c->norm + 5, c->x0);
    c->launches++;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
        e = forward(c, npts, true);
    if (e == cudaSuccess)
        e = backward(c, xs, ts, nf, batch);
    double l = 0;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&l, c->loss, 8, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess)
        return ccuda(c, e, "cnn gradients");
    if (loss)
        *loss = l / ((double)NC * npts);
    return grads ? unpack(c, c->g, grads) : GBFD_OK;
}

gbfd_status gbfd_cnn_train_step(gbfd_cnn *c, const float *xs, const float *ts, int nf, int batch,
                                float lr, double *loss)
{
    gbfd_status st = check(c, batch);
    if (st != GBFD_OK)
        return st;
    if (!xs || !ts || (nf != 4 && nf != 5) || !(lr >= 0)) {
        cerr(c, "cnn train_step: bad arguments");
        return GBFD_ERR_INVALID_ARG;
    }
    const int n3 = c->n * c->n * c->n, npts = batch * n3;
    k_input_compact<<<(npts + 255) / 256, 256, 0, c->stream>>>(xs, nf, c->n, npts, c->batch,
                                                                c->norm, c->norm + 5, c->x0);
    c->launches++;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
        e = forward(c, npts, true);
    if (e == cudaSuccess)
        e = backward(c, xs, ts, nf, batch);
    c->adam_t++;
    if (e == cudaSuccess)
        e = pack(c, c->g, lr);
    if (e == cudaSuccess && loss) {
        double l = 0;
        e = cudaMemcpyAsync(&l, c->loss, 8, cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess)
            e = cudaStreamSynchronize(c->stream);
        *loss = l / ((double)NC * npts);
    }
    return e == cudaSuccess ? GBFD_OK : ccuda(c, e, "cnn train_step");
}

gbfd_status gbfd_cnn_apply(gbfd_cnn *c, gbfd_ctx *ctx)
{
    if (!c || !ctx)
        return GBFD_ERR_INVALID_ARG;
    float *st = nullptr;
    Layout L;
    int nf = 0;
    cudaStream_t s;
    if (!ctx_view(ctx, &st, &L, &nf, &s)) {
        cerr(c, "cnn apply: context must be FP32 with a cubic grid");
        return GBFD_ERR_UNSUPPORTED;
    }
    if (L.nx != c->n) {
        cerr(c, "cnn apply: grid %d does not match the network's %d", L.nx, c->n);
        return GBFD_ERR_INVALID_ARG;
    }
    const int n3 = c->n * c->n * c->n;
    // run on the solver's stream so the correction is ordered with its steps
    const cudaStream_t saved = c->stream;
    c->stream = s;
    k_input_state<<<(n3 + 255) / 256, 256, 0, s>>>(st, L, nf, c->batch, c->norm, c->norm + 5,
                                                   c->x0);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
        e = forward(c, n3, false);
    if (e == cudaSuccess) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((n3 + 255) / 256);
        cfg.blockDim = dim3(256);
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        e = cudaLaunchKernelEx(&cfg, k_apply, st, L, nf, (const float *)c->y3,
                               (const float *)(c->norm + 10));
        if (e == cudaSuccess)
            e = cudaGetLastError();
    }
    c->stream = saved;
    c->launches += 2;
    return e == cudaSuccess ? GBFD_OK : ccuda(c, e, "cnn apply");
}

gbfd_status gbfd_step_corrected(gbfd_ctx *ctx, gbfd_cnn *c, double dt, int nsteps)
{
    if (!ctx || !c || nsteps < 0)
        return GBFD_ERR_INVALID_ARG;
    for (int i = 0; i < nsteps; ++i) {
        gbfd_status st = gbfd_rk3_step(ctx, dt, 1);
        if (st != GBFD_OK)
            return st;
        st = gbfd_cnn_apply(c, ctx);
        if (st != GBFD_OK)
            return st;
    }
    return GBFD_OK;
}

gbfd_status gbfd_box_filter(gbfd_ctx *fine, int r, float *out)
{
    float *st = nullptr;
    Layout L;
    int nf = 0;
    cudaStream_t s;
    if (!fine || !out || r < 2 || r % 2)
        return GBFD_ERR_INVALID_ARG;
    if (!ctx_view(fine, &st, &L, &nf, &s) || L.nx % r)
        return GBFD_ERR_UNSUPPORTED;
    const int nc = L.nx / r;
    const long long cnt = (long long)nc * nc * nc * nf;
    k_box_filter<<<(unsigned)((cnt + 255) / 256), 256, 0, s>>>(st, L, nf, r, out);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GBFD_OK : GBFD_ERR_CUDA;
}

int64_t gbfd_cnn_launch_count(const gbfd_cnn *c) { return c ? c->launches : 0; }

const char *gbfd_cnn_last_error(const gbfd_cnn *c) { return c ? c->err : g_cnn_err; }

}  // extern "C"
