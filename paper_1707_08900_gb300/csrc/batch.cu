// Batched form: many independent periodic cubic boxes of uneven sizes, each
// with its own viscosity and time step, advanced together.  The work is a
// list of equal-cost columns (box, tile, z-chunk) drawn from all boxes, each
// streamed through the same TMA-staged two-points-per-thread pipeline as the
// single-box kernels (the two-plane packed column routine on 32 x 8 or 64 x 8
// tiles, or the lagged-output routine with its pending right-hand sides in
// TMEM on 32 x 8 tiles), FP32 storage and arithmetic.  Two ways to run it:
//
// * dataflow (the default): ALL substeps of a run of RK3 steps in ONE
//   persistent launch.  CTAs take work items (substep k, column i) in order
//   from an atomic counter; an item of box b at substep k waits (bounded)
//   until the box's completion counter shows every column of its substeps
//   before k done, then streams its column and adds one to the counter
//   (release after the stores, acquire before the TMA loads).  Items are
//   taken in order and only wait for items taken earlier, so the launch
//   cannot deadlock whatever the residency; boxes at different substeps
//   overlap, so no device-wide barrier is ever needed;
// * one persistent launch per substep walking the list (CTAs stride it).
//
// A run of RK3 steps is captured once as a CUDA graph and replayed.  Per-box
// data lives in device memory: the TMA descriptors of the box's two state
// buffers and its u-tilde (for both tile widths), the buffer pointers and
// layout, and the stencil weights with the box's spacing folded in (cubic
// cells: one set of weights for all axes; the lagged routine reads them from
// shared memory, where they do not cost registers).  Time steps are read
// from a device array the host refreshes before each replay, so one graph
// serves any dt.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <utility>
#include <vector>

#include "../../include/gbfd.h"
#include "tiled4_impl.cuh"

namespace gbfd {
namespace batch {

constexpr int NS = 8, U = 2;  // ring slots, output planes per loop iteration

// Column routines (kernel kinds) and their tiles.
enum { KIND_PACKED = 0, KIND_LAG = 1, KIND_PACKED64 = 2, NKIND = 3 };
__host__ __device__ constexpr int kind_tx(int kind) { return kind == KIND_PACKED64 ? 64 : 32; }
constexpr int TY = 8;

struct BoxDesc {
    CUtensorMap tm_state[2][2];  // [tile width 32 / 64][buffer]: halo boxes of the state
    CUtensorMap tm_w[2];         // [tile width]: tile boxes of u-tilde
    float *state[2];             // origins of the padded state buffers
    float *w;                    // origin of the padded u-tilde buffer
    Layout L;                    // layout of all three (FP32)
    CubicCoef<float> coef;
    int nitems;                  // columns of this box in the work list
};

// Device-side state of the dataflow launch, zeroed before each launch.
struct Flow {
    int next;   // next work item to hand out
    int abort;  // a wait gave up: stop taking work
    int done[1];  // [nbox] columns completed, over all substeps so far
};

template <int KIND, int NF>
constexpr int smem_bytes()
{
    if constexpr (KIND == KIND_LAG)
        return tiled4::RingL<float, NF, 32, TY, NS, U>::BYTES;
    else
        return tiled2::Ring<float, float, NF, kind_tx(KIND), TY, NS, U + 2>::BYTES;
}

// One column of one box at substep s (parity: which state buffer is the
// input).  Returns false when a bounded wait gave up.
// SPEC: boxes on whole tiles take one instantiation of the column routine
// per RK3 substep (two-plane routine, five fields), as the single-box kernels
// do; the substep and the grid-extent test then leave the per-plane code.
template <int KIND, int NF, bool SPEC = false>
__device__ __forceinline__ bool run_item(const BoxDesc *__restrict__ B, const int4 item,
                                         const int s, const int parity, const float dt,
                                         const int zc, const CubicCoef<float> &scoef, int &jrun,
                                         int &wrun, unsigned char *smem, int *dev_error,
                                         const uint32_t tmem)
{
    constexpr int TX = kind_tx(KIND);
    constexpr int wi = TX == 64 ? 1 : 0;
    const Layout L = B->L;
    const int nout = min(zc, L.nz - item.w);
    // Williamson's coefficients (common.cuh: RK3_ALPHA, RK3_BETA), in FP32
    const float alpha = s == 0 ? 0.0f : (s == 1 ? (float)(-5.0 / 9.0) : (float)(-153.0 / 128.0));
    const float beta = s == 0 ? (float)(1.0 / 3.0) : (s == 1 ? (float)(15.0 / 16.0)
                                                            : (float)(8.0 / 15.0));
    if constexpr (KIND == KIND_LAG) {
        return tiled4::run_column<float, float, NF, TX, TY, NS, U, false, false, true>(
            &B->tm_state[wi][parity], &B->tm_w[wi], B->state[parity ^ 1], B->w, L, L, scoef,
            alpha, beta, dt, s == 0, s == 2, item.y, item.z, item.w, nout, jrun, wrun, smem,
            dev_error, -1, nullptr, tmem);
    } else {
        const CubicCoef<float> c = B->coef;
        if constexpr (SPEC && NF == 5) {
            if (L.nx % TX == 0 && L.ny % TY == 0) {
                auto run = [&](auto stg) {
                    constexpr int S = decltype(stg)::value;
                    return tiled2::run_column<float, float, float, NF, true, TX, TY, NS, true, U,
                                              false, false, false, CubicCoef<float>, S, true>(
                        &B->tm_state[wi][parity], &B->tm_w[wi], B->state[parity ^ 1], B->w,
                        nullptr, L, L, c, alpha, beta, dt, S == 0, S == 2, item.y, item.z, item.w,
                        nout, jrun, wrun, smem, dev_error);
                };
                if (s == 0)
                    return run(std::integral_constant<int, 0>{});
                if (s == 1)
                    return run(std::integral_constant<int, 1>{});
                return run(std::integral_constant<int, 2>{});
            }
        }
        return tiled2::run_column<float, float, float, NF, true, TX, TY, NS, true, U, false>(
            &B->tm_state[wi][parity], &B->tm_w[wi], B->state[parity ^ 1], B->w, nullptr, L, L, c,
            alpha, beta, dt, s == 0, s == 2, item.y, item.z, item.w, nout, jrun, wrun, smem,
            dev_error);
    }
}

template <int KIND>
__device__ __forceinline__ uint32_t tmem_open(unsigned char *smem, int bytes)
{
    if constexpr (KIND != KIND_LAG)
        return 0;
    uint32_t *slot = reinterpret_cast<uint32_t *>(smem + bytes - 16);
    if (threadIdx.x < 32)
        tc::tmem_alloc(slot, tiled4::kTmCols);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    return *reinterpret_cast<volatile uint32_t *>(slot);
}

template <int KIND>
__device__ __forceinline__ void tmem_close(uint32_t tmem)
{
    if constexpr (KIND == KIND_LAG) {
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        if (threadIdx.x < 32)
            tc::tmem_dealloc(tmem, tiled4::kTmCols);
    }
}

// One persistent launch per substep: the CTAs stride the work list.
template <int KIND, int NF>
__global__ void __launch_bounds__((kind_tx(KIND) / 2) * TY) k_batch_substep(
    const BoxDesc *__restrict__ boxes, const int4 *__restrict__ items, const int nitems,
    const float *__restrict__ dts, const int zc, const int s, const int parity,
    int *__restrict__ dev_error)
{
    constexpr int SMB = smem_bytes<KIND, NF>();
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ CubicCoef<float> scoef;
    if constexpr (KIND == KIND_LAG)
        tiled2::init_barriers(reinterpret_cast<uint64_t *>(
                                  smem + tiled4::RingL<float, NF, 32, TY, NS, U>::BAR_OFF),
                              NS + U + 2);
    else
        tiled2::init_barriers(reinterpret_cast<uint64_t *>(
                                  smem + tiled2::Ring<float, float, NF, kind_tx(KIND), TY, NS,
                                                      U + 2>::BAR_OFF),
                              NS + U + 2);
    const uint32_t tmem = tmem_open<KIND>(smem, SMB);
    int jrun = 0, wrun = 0;
#pragma unroll 1
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const int4 item = items[it];  // box, x0, y0, z0
        const BoxDesc *B = boxes + item.x;
        __syncthreads();  // every thread is done with the previous box's weights
        if (threadIdx.x == 0)
            scoef = B->coef;
        __syncthreads();
        if (!run_item<KIND, NF>(B, item, s, parity, dts[item.x], zc, scoef, jrun, wrun, smem,
                                dev_error, tmem))
            break;
    }
    tmem_close<KIND>(tmem);
}

__device__ __forceinline__ int ld_acquire(const int *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// All substeps of nsub = 3 nsteps in one persistent launch (dataflow over
// per-box completion counters; see the top of the file).  stall_item (tests
// only, -1 = off): the CTA that finishes this work item does not count it,
// so the items that depend on it wait until their bounded wait gives up.
template <int KIND, int NF>
__global__ void __launch_bounds__((kind_tx(KIND) / 2) * TY) k_batch_flow(
    const BoxDesc *__restrict__ boxes, const int4 *__restrict__ items, const int nitems,
    const int nsub, const float *__restrict__ dts, const int zc, const int cur,
    Flow *__restrict__ flow, int *__restrict__ dev_error, const int stall_item)
{
    constexpr int SMB = smem_bytes<KIND, NF>();
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ CubicCoef<float> scoef;
    __shared__ int sq;
    if constexpr (KIND == KIND_LAG)
        tiled2::init_barriers(reinterpret_cast<uint64_t *>(
                                  smem + tiled4::RingL<float, NF, 32, TY, NS, U>::BAR_OFF),
                              NS + U + 2);
    else
        tiled2::init_barriers(reinterpret_cast<uint64_t *>(
                                  smem + tiled2::Ring<float, float, NF, kind_tx(KIND), TY, NS,
                                                      U + 2>::BAR_OFF),
                              NS + U + 2);
    const uint32_t tmem = tmem_open<KIND>(smem, SMB);
    const long long nq = (long long)nsub * nitems;
    int jrun = 0, wrun = 0;
#pragma unroll 1
    while (true) {
        if (threadIdx.x == 0) {
            int q = -1;
            if (!ld_acquire(&flow->abort)) {
                q = atomicAdd(&flow->next, 1);
                if (q < nq) {
                    const int k = q / nitems;
                    const int box = items[q % nitems].x;
                    // every column of this box's substeps before k is done
                    const int need = k * boxes[box].nitems;
                    if (ld_acquire(&flow->done[box]) < need) {
                        const uint64_t t0 = tiled::global_ns();
                        while (ld_acquire(&flow->done[box]) < need) {
                            if (ld_acquire(&flow->abort) ||
                                tiled::global_ns() - t0 > 2000000000ull) {
                                atomicExch(&flow->abort, 1);
                                atomicExch(dev_error, 3);
                                q = -1;
                                break;
                            }
                            __nanosleep(256);
                        }
                    }
                    // the other CTAs' generic-proxy stores are visible: order
                    // them before this thread's TMA (async-proxy) loads
                    asm volatile("fence.proxy.async.global;" ::: "memory");
                } else {
                    q = -1;
                }
            }
            sq = q;
            if (q >= 0)
                scoef = boxes[items[q % nitems].x].coef;
        }
        __syncthreads();
        const int q = sq;
        if (q < 0)
            break;
        const int k = q / nitems;
        const int4 item = items[q % nitems];
        const BoxDesc *B = boxes + item.x;
        const bool ok = run_item<KIND, NF, KIND == KIND_PACKED>(B, item, k % 3, (cur + k) & 1,
                                                               dts[item.x], zc, scoef, jrun, wrun,
                                                               smem, dev_error, tmem);
        __syncthreads();  // the column's stores are issued by every thread
        if (threadIdx.x == 0) {
            if (!ok)
                atomicExch(&flow->abort, 1);
            else if (q != stall_item) {
                __threadfence();  // release: the stores before the count
                atomicAdd(&flow->done[item.x], 1);
            }
        }
        if (!ok)
            break;
    }
    tmem_close<KIND>(tmem);
}

// CTAs of a kernel that fit on one SM by its registers, shared memory and
// threads, and by the tensor-memory columns each CTA allocates (tm_cols of
// the SM's 512; 0 = none).  The occupancy calculator gives a kernel that
// allocates tensor memory one CTA per SM (the allocation's size is not part
// of the kernel's attributes); the lagged routine takes 64 columns, so its
// registers and shared memory decide.  The persistent grids need the true
// figure: the dataflow launch is correct at any residency, but half-filled
// SMs halve its throughput.
int fit_per_sm(const void *kern, int threads, int dyn_smem, int dev, int tm_cols)
{
    cudaFuncAttributes fa;
    int regs_sm = 0, smem_sm = 0, smem_res = 0, thr_sm = 0;
    if (cudaFuncGetAttributes(&fa, kern) != cudaSuccess ||
        cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev) !=
            cudaSuccess ||
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) !=
            cudaSuccess ||
        cudaDeviceGetAttribute(&smem_res, cudaDevAttrReservedSharedMemoryPerBlock, dev) !=
            cudaSuccess ||
        cudaDeviceGetAttribute(&thr_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev) != cudaSuccess)
        return 0;
    const int warps = (threads + 31) / 32;
    const int regs_warp = (fa.numRegs * 32 + 255) / 256 * 256;  // allocated per warp in 256s
    const int smem_cta = (dyn_smem + (int)fa.sharedSizeBytes + smem_res + 127) / 128 * 128;
    int per = thr_sm / threads;
    if (regs_warp > 0)
        per = std::min(per, regs_sm / (regs_warp * warps));
    if (smem_cta > 0)
        per = std::min(per, smem_sm / smem_cta);
    if (tm_cols > 0)
        per = std::min(per, 512 / tm_cols);
    return per;
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

bool encode(CUtensorMap *m, const void *origin, const Layout &L, int nf, int bx, int by)
{
    PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
    if (!fn)
        return false;
    const cuuint64_t dims[4] = {(cuuint64_t)(L.nx + 2 * GX), (cuuint64_t)L.rows,
                                (cuuint64_t)L.nz, (cuuint64_t)nf};
    const cuuint64_t strides[3] = {(cuuint64_t)(L.P * L.w), (cuuint64_t)(L.plane * L.w),
                                   (cuuint64_t)(L.fpitch * L.w)};
    const cuuint32_t box[4] = {(cuuint32_t)bx, (cuuint32_t)by, 1u, (cuuint32_t)nf};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<void *>(origin), dims, strides,
              box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

struct Plan {
    std::vector<Layout> lay;
    std::vector<size_t> off_state0, off_state1, off_w;
    size_t off_desc, off_items, off_dt, off_staging, off_part, off_out, off_err, off_flow, total;
    int nitems;
    int ndiag;
};

size_t flow_bytes(int nbox) { return sizeof(int) * (2 + (size_t)nbox); }

int zc_for(int n, int zc) { return std::min(zc, n); }

int count_items(const int32_t *n, int nbox, int zc, int tx)
{
    int c = 0;
    for (int b = 0; b < nbox; ++b) {
        const int z = zc_for(n[b], zc);
        c += ((n[b] + tx - 1) / tx) * ((n[b] + TY - 1) / TY) * ((n[b] + z - 1) / z);
    }
    return c;
}


bool make_plan(int nbox, const int32_t *n, int entropy_mode, Plan &pl, char *why, size_t wn)
{
    if (nbox < 1 || nbox > 4096 || !n) {
        snprintf(why, wn, "nbox must be in 1..4096 and n non-NULL");
        return false;
    }
    const int nf = entropy_mode ? 5 : 4;
    size_t off = 0;
    long long maxpts = 0;
    pl.lay.resize(nbox);
    pl.off_state0.resize(nbox);
    pl.off_state1.resize(nbox);
    pl.off_w.resize(nbox);
    for (int b = 0; b < nbox; ++b) {
        if (n[b] < 8 || n[b] % 4 || n[b] > 1024) {
            snprintf(why, wn, "box %d: n = %d must be a multiple of 4 in 8..1024", b, n[b]);
            return false;
        }
        pl.lay[b] = make_layout(n[b], n[b], n[b], 4, nf);
        pl.off_state0[b] = off;
        off = align256(off + pl.lay[b].bytes);
        pl.off_state1[b] = off;
        off = align256(off + pl.lay[b].bytes);
        pl.off_w[b] = off;
        off = align256(off + pl.lay[b].bytes);
        maxpts = std::max(maxpts, (long long)n[b] * n[b] * n[b]);
    }
    pl.off_desc = off;
    off = align256(off + sizeof(BoxDesc) * nbox);
    // the work list is sized for the smallest z-chunk (8) and tile (32 wide)
    pl.nitems = count_items(n, nbox, 8, 32);
    pl.off_items = off;
    off = align256(off + sizeof(int4) * pl.nitems);
    pl.off_dt = off;
    off = align256(off + sizeof(float) * nbox);
    pl.off_staging = off;
    off = align256(off + (size_t)nf * maxpts * 8);
    pl.ndiag = diag_blocks(make_layout(1024, 1024, 1024, 4, nf));
    pl.off_part = off;
    off = align256(off + (size_t)pl.ndiag * 16 * sizeof(double));
    pl.off_out = off;
    off = align256(off + 16 * sizeof(double));
    pl.off_err = off;
    off = align256(off + 256);
    pl.off_flow = off;
    off = align256(off + flow_bytes(nbox));
    pl.total = off;
    return true;
}

}  // namespace batch
}  // namespace gbfd

using namespace gbfd;
using namespace gbfd::batch;

struct gbfd_batch {
    int nbox, nf;
    cudaStream_t stream, cap;
    char *ws;
    Plan plan;
    std::vector<int> n;
    std::vector<double> L, nu;
    double cs;
    std::vector<BoxDesc> hdesc;
    BoxDesc *ddesc;
    int4 *ditems;
    float *ddt;
    char *staging;
    double *dpart, *dout;
    int *derr;
    Flow *dflow;
    int cur;
    int zc;
    int kind;        // column routine (KIND_*)
    int flow;        // 1: all substeps in one dataflow launch; 0: one launch per substep
    int stall_item;  // tests: a work item whose completion is never counted (-1 off)
    int grid;        // CTAs of a launch (0: resident CTAs of the kind on every SM)
    int grid_kind[NKIND];
    int use_graph;
    int nitems;
    int64_t launches;
    std::map<std::pair<int, int>, cudaGraphExec_t> graphs;
    char err[512];
};

namespace {

thread_local char g_batch_err[512];

void berr(gbfd_batch *b, const char *fmt, ...)
{
    char *buf = b ? b->err : g_batch_err;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, 512, fmt, ap);
    va_end(ap);
}

gbfd_status bcuda(gbfd_batch *b, cudaError_t e, const char *what)
{
    berr(b, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
    return GBFD_ERR_CUDA;
}

void drop_graphs(gbfd_batch *b)
{
    for (auto &kv : b->graphs)
        cudaGraphExecDestroy(kv.second);
    b->graphs.clear();
}

// Build the work list for chunk length zc and the kind's tile: box-major so
// that neighbouring CTAs stream neighbouring tiles of the same box (halo
// reuse in L2); each box's column count goes to its descriptor (the dataflow
// launch's completion target).
gbfd_status build_items(gbfd_batch *b, int zc, int kind)
{
    std::vector<int4> items;
    const int tx = kind_tx(kind);
    for (int bx = 0; bx < b->nbox; ++bx) {
        const int n = b->n[bx];
        const int z = zc_for(n, zc);
        const size_t before = items.size();
        for (int z0 = 0; z0 < n; z0 += z)
            for (int y0 = 0; y0 < n; y0 += TY)
                for (int x0 = 0; x0 < n; x0 += tx)
                    items.push_back(make_int4(bx, x0, y0, z0));
        b->hdesc[bx].nitems = (int)(items.size() - before);
    }
    if ((int)items.size() > b->plan.nitems) {
        berr(b, "work list overflow");
        return GBFD_ERR_INVALID_ARG;
    }
    cudaError_t e = cudaMemcpyAsync(b->ditems, items.data(), sizeof(int4) * items.size(),
                                    cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->ddesc, b->hdesc.data(), sizeof(BoxDesc) * b->nbox,
                            cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess)
        return bcuda(b, e, "work list upload");
    b->nitems = (int)items.size();
    b->zc = zc;
    b->kind = kind;
    drop_graphs(b);
    return GBFD_OK;
}

int grid_of(const gbfd_batch *b) { return b->grid > 0 ? b->grid : b->grid_kind[b->kind]; }

template <int KIND, int NF>
cudaError_t launch_substep_k(gbfd_batch *b, int s, int parity, cudaStream_t stream)
{
    k_batch_substep<KIND, NF><<<grid_of(b), (kind_tx(KIND) / 2) * TY, smem_bytes<KIND, NF>(),
                                stream>>>(b->ddesc, b->ditems, b->nitems, b->ddt, b->zc, s, parity,
                                          b->derr);
    return cudaGetLastError();
}

template <int KIND, int NF>
cudaError_t launch_flow_k(gbfd_batch *b, int nsub, int cur, cudaStream_t stream)
{
    cudaError_t e = cudaMemsetAsync(b->dflow, 0, flow_bytes(b->nbox), stream);
    if (e != cudaSuccess)
        return e;
    k_batch_flow<KIND, NF><<<grid_of(b), (kind_tx(KIND) / 2) * TY, smem_bytes<KIND, NF>(),
                             stream>>>(b->ddesc, b->ditems, b->nitems, nsub, b->ddt, b->zc, cur,
                                       b->dflow, b->derr, b->stall_item);
    return cudaGetLastError();
}

#define GBFD_BATCH_DISPATCH(FN, ...)                                                              \
    (b->nf == 5 ? (b->kind == KIND_LAG      ? FN<KIND_LAG, 5>(__VA_ARGS__)                        \
                   : b->kind == KIND_PACKED64 ? FN<KIND_PACKED64, 5>(__VA_ARGS__)                 \
                                              : FN<KIND_PACKED, 5>(__VA_ARGS__))                  \
                : (b->kind == KIND_LAG      ? FN<KIND_LAG, 4>(__VA_ARGS__)                        \
                   : b->kind == KIND_PACKED64 ? FN<KIND_PACKED64, 4>(__VA_ARGS__)                 \
                                              : FN<KIND_PACKED, 4>(__VA_ARGS__)))

cudaError_t launch_one(gbfd_batch *b, int s, int parity, cudaStream_t stream)
{
    return GBFD_BATCH_DISPATCH(launch_substep_k, b, s, parity, stream);
}

// nsteps RK3 steps from state buffer `cur`: one dataflow launch, or 3 nsteps
// substep launches; returns the number of kernel launches in `nl`.
gbfd_status enqueue_steps(gbfd_batch *b, int nsteps, int cur, cudaStream_t stream, int *nl)
{
    if (b->flow) {
        cudaError_t e = GBFD_BATCH_DISPATCH(launch_flow_k, b, 3 * nsteps, cur, stream);
        if (e != cudaSuccess)
            return bcuda(b, e, "batch dataflow launch");
        *nl = 1;
        return GBFD_OK;
    }
    for (int k = 0; k < 3 * nsteps; ++k) {
        cudaError_t e = launch_one(b, k % 3, (cur + k) & 1, stream);
        if (e != cudaSuccess)
            return bcuda(b, e, "batch substep launch");
    }
    *nl = 3 * nsteps;
    return GBFD_OK;
}

gbfd_status graph_for(gbfd_batch *b, int nsteps, cudaGraphExec_t *out, int *nl)
{
    auto key = std::make_pair(nsteps, b->cur);
    auto it = b->graphs.find(key);
    *nl = b->flow ? 1 : 3 * nsteps;
    if (it != b->graphs.end()) {
        *out = it->second;
        return GBFD_OK;
    }
    cudaError_t e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess)
        return bcuda(b, e, "graph capture begin");
    int n = 0;
    gbfd_status st = enqueue_steps(b, nsteps, b->cur, b->cap, &n);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(b->cap, &g);
    if (st != GBFD_OK) {
        if (g)
            cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess)
        return bcuda(b, e, "graph capture end");
    cudaGraphExec_t ex = nullptr;
    e = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess)
        return bcuda(b, e, "graph instantiate");
    b->graphs[key] = ex;
    *out = ex;
    return GBFD_OK;
}

gbfd_status check_box(gbfd_batch *b, int box)
{
    if (!b)
        return GBFD_ERR_INVALID_ARG;
    if (box < 0 || box >= b->nbox) {
        berr(b, "box %d out of range 0..%d", box, b->nbox - 1);
        return GBFD_ERR_INVALID_ARG;
    }
    return GBFD_OK;
}

char *state_origin(gbfd_batch *b, int box, int which)
{
    const size_t off = which ? b->plan.off_state1[box] : b->plan.off_state0[box];
    return b->ws + off + b->plan.lay[box].origin;
}

}  // namespace

extern "C" {

size_t gbfd_batch_workspace_bytes(int nbox, const int32_t *n, int entropy_mode)
{
    Plan pl;
    char why[256];
    if (entropy_mode != 0 && entropy_mode != 1)
        return 0;
    if (!make_plan(nbox, n, entropy_mode, pl, why, sizeof why))
        return 0;
    return pl.total;
}

gbfd_status gbfd_batch_init(int nbox, const int32_t *n, const double *lengths, const double *nu,
                            double cs, int entropy_mode, void *workspace, size_t workspace_bytes,
                            void *stream, gbfd_batch **out)
{
    if (!out || !lengths || !nu) {
        berr(nullptr, "out, lengths and nu must be non-NULL");
        return GBFD_ERR_INVALID_ARG;
    }
    *out = nullptr;
    if (entropy_mode != 0 && entropy_mode != 1) {
        berr(nullptr, "entropy_mode must be 0 or 1");
        return GBFD_ERR_INVALID_ARG;
    }
    Plan pl;
    char why[256];
    if (!make_plan(nbox, n, entropy_mode, pl, why, sizeof why)) {
        berr(nullptr, "%s", why);
        return GBFD_ERR_INVALID_ARG;
    }
    if (!(cs >= 0) || !std::isfinite(cs)) {
        berr(nullptr, "cs must be finite and >= 0");
        return GBFD_ERR_INVALID_ARG;
    }
    for (int b = 0; b < nbox; ++b)
        if (!(lengths[b] > 0) || !std::isfinite(lengths[b]) || !(nu[b] >= 0) ||
            !std::isfinite(nu[b])) {
            berr(nullptr, "box %d: length must be > 0 and nu >= 0, both finite", b);
            return GBFD_ERR_INVALID_ARG;
        }
    if (!workspace || ((uintptr_t)workspace & 255)) {
        berr(nullptr, "workspace must be a non-NULL, 256-byte aligned device pointer");
        return GBFD_ERR_WORKSPACE;
    }
    if (workspace_bytes < pl.total) {
        berr(nullptr, "workspace has %zu bytes, %zu needed", workspace_bytes, pl.total);
        return GBFD_ERR_WORKSPACE;
    }
    gbfd_batch *b = new (std::nothrow) gbfd_batch();
    if (!b) {
        berr(nullptr, "out of host memory");
        return GBFD_ERR_INVALID_ARG;
    }
    b->nbox = nbox;
    b->nf = entropy_mode ? 5 : 4;
    b->stream = (cudaStream_t)stream;
    b->ws = (char *)workspace;
    b->plan = pl;
    b->n.assign(n, n + nbox);
    b->L.assign(lengths, lengths + nbox);
    b->nu.assign(nu, nu + nbox);
    b->cs = cs;
    b->ddesc = (BoxDesc *)(b->ws + pl.off_desc);
    b->ditems = (int4 *)(b->ws + pl.off_items);
    b->ddt = (float *)(b->ws + pl.off_dt);
    b->staging = b->ws + pl.off_staging;
    b->dpart = (double *)(b->ws + pl.off_part);
    b->dout = (double *)(b->ws + pl.off_out);
    b->derr = (int *)(b->ws + pl.off_err);
    b->cur = 0;
    b->use_graph = 1;
    b->launches = 0;
    b->err[0] = 0;
    cudaError_t e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        bcuda(nullptr, e, "capture stream");
        delete b;
        return GBFD_ERR_CUDA;
    }
    e = cudaMemsetAsync(b->ws, 0, pl.total, b->stream);
    b->hdesc.resize(nbox);
    for (int i = 0; i < nbox && e == cudaSuccess; ++i) {
        BoxDesc &d = b->hdesc[i];
        memset(&d, 0, sizeof d);
        d.L = pl.lay[i];
        d.state[0] = (float *)(b->ws + pl.off_state0[i] + d.L.origin);
        d.state[1] = (float *)(b->ws + pl.off_state1[i] + d.L.origin);
        d.w = (float *)(b->ws + pl.off_w[i] + d.L.origin);
        d.coef = make_cubic_coef<float>(lengths[i] / n[i], cs, nu[i]);
        bool ok = true;
        for (int wi = 0; wi < 2; ++wi) {
            const int tx = wi ? 64 : 32;
            ok = ok && encode(&d.tm_state[wi][0], d.state[0], d.L, b->nf, tx + 2 * GX, TY + 2 * GY) &&
                 encode(&d.tm_state[wi][1], d.state[1], d.L, b->nf, tx + 2 * GX, TY + 2 * GY) &&
                 encode(&d.tm_w[wi], d.w, d.L, b->nf, tx, TY);
        }
        if (!ok) {
            berr(nullptr, "TMA descriptor encoding failed for box %d", i);
            cudaStreamDestroy(b->cap);
            delete b;
            return GBFD_ERR_CUDA;
        }
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->ddesc, b->hdesc.data(), sizeof(BoxDesc) * nbox,
                            cudaMemcpyHostToDevice, b->stream);
    b->dflow = (Flow *)(b->ws + pl.off_flow);
    b->zc = 32;
    b->kind = KIND_PACKED;
    b->flow = 1;
    b->stall_item = -1;
    b->grid = 0;
    int dev = 0, sms = 0;
    if (e == cudaSuccess)
        e = cudaGetDevice(&dev);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // resident CTAs per SM of each kind (the persistent grids), and the
    // shared-memory limits of every kernel
    auto setup = [&](auto sub, auto flowk, int threads, int smb, int kind) {
        int per = 0;
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(sub, cudaFuncAttributeMaxDynamicSharedMemorySize, smb);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(flowk, cudaFuncAttributeMaxDynamicSharedMemorySize, smb);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, flowk, threads, smb);
        if (e == cudaSuccess && kind == KIND_LAG)
            per = std::max(per, fit_per_sm((const void *)flowk, threads, smb, dev,
                                           tiled4::kTmCols));
        b->grid_kind[kind] = sms * std::max(per, 1);
    };
    if (b->nf == 5) {
        setup(k_batch_substep<KIND_PACKED, 5>, k_batch_flow<KIND_PACKED, 5>, 128,
              smem_bytes<KIND_PACKED, 5>(), KIND_PACKED);
        setup(k_batch_substep<KIND_LAG, 5>, k_batch_flow<KIND_LAG, 5>, 128,
              smem_bytes<KIND_LAG, 5>(), KIND_LAG);
        setup(k_batch_substep<KIND_PACKED64, 5>, k_batch_flow<KIND_PACKED64, 5>, 256,
              smem_bytes<KIND_PACKED64, 5>(), KIND_PACKED64);
    } else {
        setup(k_batch_substep<KIND_PACKED, 4>, k_batch_flow<KIND_PACKED, 4>, 128,
              smem_bytes<KIND_PACKED, 4>(), KIND_PACKED);
        setup(k_batch_substep<KIND_LAG, 4>, k_batch_flow<KIND_LAG, 4>, 128,
              smem_bytes<KIND_LAG, 4>(), KIND_LAG);
        setup(k_batch_substep<KIND_PACKED64, 4>, k_batch_flow<KIND_PACKED64, 4>, 256,
              smem_bytes<KIND_PACKED64, 4>(), KIND_PACKED64);
    }
    if (e != cudaSuccess) {
        bcuda(nullptr, e, "batch init");
        cudaStreamDestroy(b->cap);
        delete b;
        return GBFD_ERR_CUDA;
    }
    gbfd_status st = build_items(b, 32, KIND_PACKED);
    if (st != GBFD_OK) {
        berr(nullptr, "%s", b->err);
        cudaStreamDestroy(b->cap);
        delete b;
        return st;
    }
    *out = b;
    return GBFD_OK;
}

gbfd_status gbfd_batch_destroy(gbfd_batch *b)
{
    if (!b)
        return GBFD_OK;
    drop_graphs(b);
    cudaStreamDestroy(b->cap);
    delete b;
    return GBFD_OK;
}

gbfd_status gbfd_batch_set_state(gbfd_batch *b, int box, const void *src, int src_on_device,
                                 int src_is_fp64)
{
    gbfd_status st = check_box(b, box);
    if (st != GBFD_OK)
        return st;
    if (!src) {
        berr(b, "src is NULL");
        return GBFD_ERR_INVALID_ARG;
    }
    const Layout &Ly = b->plan.lay[box];
    const size_t bytes = (size_t)b->nf * Ly.nx * Ly.ny * Ly.nz * (src_is_fp64 ? 8 : 4);
    const void *from = src;
    cudaError_t e = cudaSuccess;
    if (!src_on_device) {
        e = cudaMemcpyAsync(b->staging, src, bytes, cudaMemcpyHostToDevice, b->stream);
        from = b->staging;
    }
    int nl = 0;
    if (e == cudaSuccess)
        e = launch_scatter(from, src_is_fp64, state_origin(b, box, b->cur), Ly, b->nf, b->stream,
                           &nl);
    if (e == cudaSuccess && !src_on_device)
        e = cudaStreamSynchronize(b->stream);  // the staging area is shared by all boxes
    b->launches += nl;
    return e == cudaSuccess ? GBFD_OK : bcuda(b, e, "batch set_state");
}

gbfd_status gbfd_batch_get_state(gbfd_batch *b, int box, void *dst, int dst_on_device,
                                 int dst_is_fp64)
{
    gbfd_status st = check_box(b, box);
    if (st != GBFD_OK)
        return st;
    if (!dst) {
        berr(b, "dst is NULL");
        return GBFD_ERR_INVALID_ARG;
    }
    const Layout &Ly = b->plan.lay[box];
    const size_t bytes = (size_t)b->nf * Ly.nx * Ly.ny * Ly.nz * (dst_is_fp64 ? 8 : 4);
    int nl = 0;
    void *to = dst_on_device ? dst : (void *)b->staging;
    cudaError_t e =
        launch_gather(state_origin(b, box, b->cur), Ly, to, dst_is_fp64, b->nf, b->stream, &nl);
    b->launches += nl;
    if (e == cudaSuccess && !dst_on_device) {
        e = cudaMemcpyAsync(dst, b->staging, bytes, cudaMemcpyDeviceToHost, b->stream);
        if (e == cudaSuccess)
            e = cudaStreamSynchronize(b->stream);
    }
    return e == cudaSuccess ? GBFD_OK : bcuda(b, e, "batch get_state");
}

gbfd_status gbfd_batch_step(gbfd_batch *b, const double *dt, int nsteps)
{
    if (!b)
        return GBFD_ERR_INVALID_ARG;
    if (!dt || nsteps < 0) {
        berr(b, "dt must be non-NULL and nsteps >= 0");
        return GBFD_ERR_INVALID_ARG;
    }
    if (nsteps == 0)
        return GBFD_OK;
    std::vector<float> h(b->nbox);
    for (int i = 0; i < b->nbox; ++i) {
        if (!(dt[i] > 0) || !std::isfinite(dt[i])) {
            berr(b, "box %d: dt %g rejected", i, dt[i]);
            return GBFD_ERR_INVALID_ARG;
        }
        h[i] = (float)dt[i];
    }
    cudaError_t e = cudaMemcpyAsync(b->ddt, h.data(), sizeof(float) * b->nbox,
                                    cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(b->stream);  // h is a local buffer
    if (e != cudaSuccess)
        return bcuda(b, e, "batch dt upload");
    gbfd_status st;
    int nl = 0;
    if (b->use_graph) {
        cudaGraphExec_t ex;
        st = graph_for(b, nsteps, &ex, &nl);
        if (st != GBFD_OK)
            return st;
        e = cudaGraphLaunch(ex, b->stream);
        if (e != cudaSuccess)
            return bcuda(b, e, "graph launch");
    } else {
        st = enqueue_steps(b, nsteps, b->cur, b->stream, &nl);
        if (st != GBFD_OK)
            return st;
    }
    b->launches += nl;
    b->cur ^= (nsteps & 1);  // 3 nsteps buffer swaps
    return GBFD_OK;
}

gbfd_status gbfd_batch_sync(gbfd_batch *b)
{
    if (!b)
        return GBFD_ERR_INVALID_ARG;
    int herr = 0;
    cudaError_t e = cudaMemcpyAsync(&herr, b->derr, sizeof(int), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess)
        return bcuda(b, e, "batch sync");
    if (herr) {
        berr(b, "device-side bounded wait gave up (code %d)", herr);
        cudaMemsetAsync(b->derr, 0, sizeof(int), b->stream);
        return GBFD_ERR_TIMEOUT;
    }
    return GBFD_OK;
}

gbfd_status gbfd_batch_diagnostics(gbfd_batch *b, int box, gbfd_diag *out)
{
    gbfd_status st = check_box(b, box);
    if (st != GBFD_OK)
        return st;
    if (!out) {
        berr(b, "out is NULL");
        return GBFD_ERR_INVALID_ARG;
    }
    const Layout &Ly = b->plan.lay[box];
    const double h = b->L[box] / b->n[box];
    int nl = 0;
    cudaError_t e = launch_diagnostics(state_origin(b, box, b->cur), Ly, b->nf, h * h * h,
                                       b->dpart, diag_blocks(Ly), b->dout, b->stream, &nl);
    b->launches += nl;
    double hv[16];
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(hv, b->dout, sizeof hv, cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess)
        return bcuda(b, e, "batch diagnostics");
    out->mass = hv[0];
    out->ekin = hv[1];
    out->umax = hv[2];
    out->urms = hv[3];
    for (int f = 0; f < 5; ++f) {
        out->rms[f] = hv[4 + f];
        out->maxabs[f] = hv[9 + f];
    }
    out->nonfinite = hv[14] != 0.0;
    out->nfields = b->nf;
    return GBFD_OK;
}

gbfd_status gbfd_batch_set_option(gbfd_batch *b, int key, int64_t value)
{
    if (!b)
        return GBFD_ERR_INVALID_ARG;
    switch (key) {
    case GBFD_BATCH_OPT_GRAPH:
        if (value != 0 && value != 1)
            break;
        b->use_graph = (int)value;
        return GBFD_OK;
    case GBFD_BATCH_OPT_ZCHUNK:
        if (value != 8 && value != 16 && value != 32 && value != 64)
            break;
        return build_items(b, (int)value, b->kind);
    case GBFD_BATCH_OPT_GRID:
        if (value < 0 || value > 65535)
            break;
        b->grid = (int)value;
        drop_graphs(b);
        return GBFD_OK;
    case GBFD_BATCH_OPT_KERNEL:
        if (value < 0 || value >= NKIND)
            break;
        return build_items(b, b->zc, (int)value);
    case GBFD_BATCH_OPT_DATAFLOW:
        if (value != 0 && value != 1)
            break;
        b->flow = (int)value;
        drop_graphs(b);
        return GBFD_OK;
    case GBFD_BATCH_OPT_FAULT_STALL:
        if (value < -1 || value > (1LL << 30))
            break;
        b->stall_item = (int)value;
        drop_graphs(b);
        return GBFD_OK;
    default:
        break;
    }
    berr(b, "batch option %d: value %lld rejected", key, (long long)value);
    return GBFD_ERR_INVALID_ARG;
}

int64_t gbfd_batch_launch_count(const gbfd_batch *b) { return b ? b->launches : 0; }

const char *gbfd_batch_last_error(const gbfd_batch *b) { return b ? b->err : g_batch_err; }

gbfd_status gbfd_batch_get_option(const gbfd_batch *b, int key, int64_t *value)
{
    if (!b || !value)
        return GBFD_ERR_INVALID_ARG;
    switch (key) {
    case GBFD_BATCH_OPT_GRAPH:
        *value = b->use_graph;
        return GBFD_OK;
    case GBFD_BATCH_OPT_ZCHUNK:
        *value = b->zc;
        return GBFD_OK;
    case GBFD_BATCH_OPT_GRID:
        *value = grid_of(b);
        return GBFD_OK;
    case GBFD_BATCH_OPT_KERNEL:
        *value = b->kind;
        return GBFD_OK;
    case GBFD_BATCH_OPT_DATAFLOW:
        *value = b->flow;
        return GBFD_OK;
    case GBFD_BATCH_OPT_FAULT_STALL:
        *value = b->stall_item;
        return GBFD_OK;
    default:
        return GBFD_ERR_INVALID_ARG;
    }
}

gbfd_status gbfd_batch_autotune(gbfd_batch *b, int steps, int *best_zc, double *best_ms)
{
    if (!b || steps < 1)
        return GBFD_ERR_INVALID_ARG;
    // Times every (column routine, z-chunk, dataflow or per-substep) on real
    // RK3 steps with dt = 0, which leave the state's values unchanged
    // (u + beta * 0 = u), and keeps the fastest.
    const int zcs[] = {8, 16, 32, 64};
    double best = 1e30;
    int bz = b->zc, bk = b->kind, bf = b->flow;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return bcuda(b, cudaGetLastError(), "autotune events");
    std::vector<float> zero(b->nbox, 0.0f);
    cudaError_t e = cudaMemcpyAsync(b->ddt, zero.data(), sizeof(float) * b->nbox,
                                    cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(b->stream);
    gbfd_status st = GBFD_OK;
    for (int kind = 0; kind < NKIND && e == cudaSuccess && st == GBFD_OK; ++kind)
        for (int zc : zcs) {
            if (e != cudaSuccess || st != GBFD_OK)
                break;
            st = build_items(b, zc, kind);
            for (int flow = 0; flow < 2 && st == GBFD_OK && e == cudaSuccess; ++flow) {
                b->flow = flow;
                int nl = 0;
                st = enqueue_steps(b, 1, b->cur, b->stream, &nl);  // warm-up
                b->launches += nl;
                b->cur ^= 1;
                if (st == GBFD_OK)
                    e = cudaEventRecord(e0, b->stream);
                if (st == GBFD_OK && e == cudaSuccess)
                    st = enqueue_steps(b, steps, b->cur, b->stream, &nl);
                b->launches += nl;
                b->cur ^= (steps & 1);
                if (st == GBFD_OK && e == cudaSuccess)
                    e = cudaEventRecord(e1, b->stream);
                if (st == GBFD_OK && e == cudaSuccess)
                    e = cudaEventSynchronize(e1);
                float ms = 0;
                if (st == GBFD_OK && e == cudaSuccess)
                    e = cudaEventElapsedTime(&ms, e0, e1);
                if (st == GBFD_OK && e == cudaSuccess && ms / steps < best) {
                    best = ms / steps;
                    bz = zc;
                    bk = kind;
                    bf = flow;
                }
            }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != GBFD_OK)
        return st;
    if (e != cudaSuccess)
        return bcuda(b, e, "autotune");
    b->flow = bf;
    st = build_items(b, bz, bk);
    if (st != GBFD_OK)
        return st;
    if (best_zc)
        *best_zc = bz;
    if (best_ms)
        *best_ms = best;
    return GBFD_OK;
}

}  // extern "C"
