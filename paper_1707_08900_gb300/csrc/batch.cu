// Batched form: many independent periodic cubic boxes of uneven sizes, each
// with its own viscosity and time step, advanced together.  Every substep is
// ONE persistent launch whose CTAs walk a work list of equal-cost columns
// (box, 32x8 tile, z-chunk) drawn from all boxes, through the same
// TMA-staged two-points-per-thread pipeline as the single-box kernel
// (tiled2::run_column, packed FP32x2 form); a run of RK3 steps is captured
// once as a CUDA graph and replayed.  FP32 storage and arithmetic.
//
// Per-box data lives in device memory: the TMA descriptors of the box's two
// state buffers and its u-tilde, the buffer pointers and layout, and the
// stencil weights with the box's spacing folded in (cubic cells: one set of
// weights for all axes, so it fits in registers).  Time steps are read from
// a device array the host refreshes before each replay, so one graph serves
// any dt.
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
#include "tiled2_impl.cuh"

namespace gbfd {
namespace batch {

constexpr int TX = 32, TY = 8, NS = 8, U = 2;  // U: output planes per loop iteration

struct BoxDesc {
    CUtensorMap tm_state[2];  // halo boxes of state buffers 0 and 1
    CUtensorMap tm_w;         // tile boxes of u-tilde
    float *state[2];          // origins of the padded state buffers
    float *w;                 // origin of the padded u-tilde buffer
    Layout L;                 // layout of all three (FP32)
    CubicCoef<float> coef;
};

template <int NF>
__global__ void __launch_bounds__((TX / 2) * TY) k_batch_substep(
    const BoxDesc *__restrict__ boxes, const int4 *__restrict__ items, const int nitems,
    const float *__restrict__ dts, const int zc, const RKStage st, const int parity,
    int *__restrict__ dev_error)
{
    using RG = tiled2::Ring<float, float, NF, TX, TY, NS, U + 2>;
    extern __shared__ __align__(128) unsigned char smem[];
    tiled2::init_barriers(reinterpret_cast<uint64_t *>(smem + RG::BAR_OFF), NS + RG::NW);
    int jrun = 0, wrun = 0;
#pragma unroll 1
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const int4 item = items[it];  // box, x0, y0, z0
        const BoxDesc *B = boxes + item.x;
        const CubicCoef<float> c = B->coef;
        const Layout L = B->L;
        const float dt = dts[item.x];
        const int nout = min(zc, L.nz - item.w);
        if (!tiled2::run_column<float, float, float, NF, true, TX, TY, NS, true, U, false>(
                &B->tm_state[parity], &B->tm_w, B->state[parity ^ 1], B->w, nullptr, L, L, c,
                (float)st.alpha, (float)st.beta, dt, st.first != 0, st.last != 0, item.y, item.z,
                item.w, nout, jrun, wrun, smem, dev_error))
            break;
    }
}

template <int NF>
constexpr int smem_bytes()
{
    return tiled2::Ring<float, float, NF, TX, TY, NS, U + 2>::BYTES;
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
    size_t off_desc, off_items, off_dt, off_staging, off_part, off_out, off_err, total;
    int nitems;
    int ndiag;
};

int zc_for(int n, int zc) { return std::min(zc, n); }

int count_items(const int32_t *n, int nbox, int zc)
{
    int c = 0;
    for (int b = 0; b < nbox; ++b) {
        const int z = zc_for(n[b], zc);
        c += ((n[b] + TX - 1) / TX) * ((n[b] + TY - 1) / TY) * ((n[b] + z - 1) / z);
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
    // the work list is sized for the smallest z-chunk offered (8)
    pl.nitems = count_items(n, nbox, 8);
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
    int cur;
    int zc;
    int grid;
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

// Build the work list for chunk length zc: box-major so that neighbouring
// CTAs stream neighbouring tiles of the same box (halo reuse in L2).
gbfd_status build_items(gbfd_batch *b, int zc)
{
    std::vector<int4> items;
    for (int bx = 0; bx < b->nbox; ++bx) {
        const int n = b->n[bx];
        const int z = zc_for(n, zc);
        for (int z0 = 0; z0 < n; z0 += z)
            for (int y0 = 0; y0 < n; y0 += TY)
                for (int x0 = 0; x0 < n; x0 += TX)
                    items.push_back(make_int4(bx, x0, y0, z0));
    }
    if ((int)items.size() > b->plan.nitems) {
        berr(b, "work list overflow");
        return GBFD_ERR_INVALID_ARG;
    }
    cudaError_t e = cudaMemcpyAsync(b->ditems, items.data(), sizeof(int4) * items.size(),
                                    cudaMemcpyHostToDevice, b->stream);
    if (e != cudaSuccess)
        return bcuda(b, e, "work list upload");
    e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess)
        return bcuda(b, e, "work list upload");
    b->nitems = (int)items.size();
    b->zc = zc;
    drop_graphs(b);
    return GBFD_OK;
}

cudaError_t launch_one(gbfd_batch *b, int s, int parity, cudaStream_t stream)
{
    RKStage st = make_stage(s, 0.0, 0.0);
    if (b->nf == 5) {
        k_batch_substep<5><<<b->grid, (TX / 2) * TY, smem_bytes<5>(), stream>>>(
            b->ddesc, b->ditems, b->nitems, b->ddt, b->zc, st, parity, b->derr);
    } else {
        k_batch_substep<4><<<b->grid, (TX / 2) * TY, smem_bytes<4>(), stream>>>(
            b->ddesc, b->ditems, b->nitems, b->ddt, b->zc, st, parity, b->derr);
    }
    return cudaGetLastError();
}

gbfd_status enqueue_steps(gbfd_batch *b, int nsteps, cudaStream_t stream)
{
    for (int k = 0; k < 3 * nsteps; ++k) {
        cudaError_t e = launch_one(b, k % 3, (b->cur + k) & 1, stream);
        if (e != cudaSuccess)
            return bcuda(b, e, "batch substep launch");
    }
    b->launches += 3 * nsteps;
    return GBFD_OK;
}

gbfd_status graph_for(gbfd_batch *b, int nsteps, cudaGraphExec_t *out)
{
    auto key = std::make_pair(nsteps, b->cur);
    auto it = b->graphs.find(key);
    if (it != b->graphs.end()) {
        *out = it->second;
        return GBFD_OK;
    }
    cudaError_t e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess)
        return bcuda(b, e, "graph capture begin");
    const int64_t before = b->launches;
    gbfd_status st = enqueue_steps(b, nsteps, b->cap);
    b->launches = before;  // counted when the graph is replayed
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
        if (!encode(&d.tm_state[0], d.state[0], d.L, b->nf, TX + 2 * GX, TY + 2 * GY) ||
            !encode(&d.tm_state[1], d.state[1], d.L, b->nf, TX + 2 * GX, TY + 2 * GY) ||
            !encode(&d.tm_w, d.w, d.L, b->nf, TX, TY)) {
            berr(nullptr, "TMA descriptor encoding failed for box %d", i);
            cudaStreamDestroy(b->cap);
            delete b;
            return GBFD_ERR_CUDA;
        }
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->ddesc, b->hdesc.data(), sizeof(BoxDesc) * nbox,
                            cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) {
        auto k5 = k_batch_substep<5>;
        auto k4 = k_batch_substep<4>;
        e = cudaFuncSetAttribute(k5, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes<5>());
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k4, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     smem_bytes<4>());
        int dev = 0, sms = 0, per = 0;
        if (e == cudaSuccess)
            e = cudaGetDevice(&dev);
        if (e == cudaSuccess)
            e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess)
            e = b->nf == 5 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                                 &per, k5, (TX / 2) * TY, smem_bytes<5>())
                           : cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                                 &per, k4, (TX / 2) * TY, smem_bytes<4>());
        b->grid = sms * std::max(per, 1);
    }
    if (e != cudaSuccess) {
        bcuda(nullptr, e, "batch init");
        cudaStreamDestroy(b->cap);
        delete b;
        return GBFD_ERR_CUDA;
    }
    gbfd_status st = build_items(b, 32);
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
    if (b->use_graph) {
        cudaGraphExec_t ex;
        st = graph_for(b, nsteps, &ex);
        if (st != GBFD_OK)
            return st;
        e = cudaGraphLaunch(ex, b->stream);
        if (e != cudaSuccess)
            return bcuda(b, e, "graph launch");
        b->launches += 3 * nsteps;
    } else {
        st = enqueue_steps(b, nsteps, b->stream);
        if (st != GBFD_OK)
            return st;
    }
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
        return build_items(b, (int)value);
    case GBFD_BATCH_OPT_GRID:
        if (value < 1 || value > 65535)
            break;
        b->grid = (int)value;
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

gbfd_status gbfd_batch_autotune(gbfd_batch *b, int steps, int *best_zc, double *best_ms)
{
    if (!b || steps < 1)
        return GBFD_ERR_INVALID_ARG;
    // time substep launches on the current state without advancing it: the
    // outputs land in the other buffer, which holds no state between steps
    const int zcs[] = {8, 16, 32, 64};
    double best = 1e30;
    int bz = b->zc;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return bcuda(b, cudaGetLastError(), "autotune events");
    std::vector<float> one(b->nbox, 1e-6f);
    cudaError_t e = cudaMemcpyAsync(b->ddt, one.data(), sizeof(float) * b->nbox,
                                    cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(b->stream);
    for (int zc : zcs) {
        if (e != cudaSuccess)
            break;
        gbfd_status st = build_items(b, zc);
        if (st != GBFD_OK) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return st;
        }
        for (int r = 0; r < steps + 1 && e == cudaSuccess; ++r) {
            if (r == 1)
                e = cudaEventRecord(e0, b->stream);
            for (int s = 0; s < 3 && e == cudaSuccess; ++s)
                e = launch_one(b, s, b->cur, b->stream);
            b->launches += 3;
        }
        if (e == cudaSuccess)
            e = cudaEventRecord(e1, b->stream);
        if (e == cudaSuccess)
            e = cudaEventSynchronize(e1);
        float ms = 0;
        if (e == cudaSuccess)
            e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && ms / steps < best) {
            best = ms / steps;
            bz = zc;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess)
        return bcuda(b, e, "autotune");
    gbfd_status st = build_items(b, bz);
    if (st != GBFD_OK)
        return st;
    if (best_zc)
        *best_zc = bz;
    if (best_ms)
        *best_ms = best;
    return GBFD_OK;
}

}  // extern "C"
