// C-ABI entry points of libgbfd (declared in include/gbfd.h): parameter
// validation, workspace carving, state copies, the RK3 step loop of
// Algorithms 2 and 3, diagnostics.  No device memory is allocated here: all
// buffers are carved from the caller's workspace.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <new>
#include <string>

#include "../../include/gbfd.h"
#include "kernels.cuh"
#include "tiled.cuh"

using namespace gbfd;

struct gbfd_ctx {
    gbfd_params p;
    int nf;
    int sbytes;  // storage bytes per value (8 FP64, 4 otherwise)
    int wbytes;  // u-tilde bytes per value
    cudaStream_t stream;
    char *ws;
    size_t ws_bytes;
    Layout Ls, Lw, Ld;
    char *state_region[2];
    char *w_region;
    char *div_region;
    char *staging;
    double *diag_part;
    double *diag_out;
    int *dev_error;  // device-side error word (bounded waits)
    int ndiag;
    int cur;         // which state buffer holds the current state
    int64_t launches;
    int kernel_path;  // 0 = tiled when supported, 1 = simple
    int tile_cfg;     // index into the tiled kernel's tile table (-1 = default)
    int sms;          // SM count of the context's device (read at init)
    double h[3];      // grid spacings (z: lz / (nz - 1) between walls)
    int fault_skip;   // test-only fault injection (-1 = off)
    int host_path;    // 0 = pinned host buffers accessed in place, 1 = always staged
    int host_async;   // 1 = gbfd_get_state to host memory does not wait for the stream
    Forcing fo;       // forcing of the step being taken (fo.on = 0: none)
    double2 *ftab;    // its per-axis phase tables (workspace)
    TmapCache tmaps;  // encoded TMA descriptors of the two state buffers
    bool broken;
    Coef<double> c64;
    Coef<float> c32;
    char err[512];
};

namespace {

thread_local char g_init_err[512];

// Device address of a pinned (page-locked) host buffer that is mapped into
// the device address space, or NULL for pageable host memory.  The copy
// kernels then read or write such a buffer in place over the CPU-GPU link,
// with no staging copy.
const void *mapped_host(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

void set_err(gbfd_ctx *c, const char *fmt, ...)
{
    char *buf = c ? c->err : g_init_err;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, 512, fmt, ap);
    va_end(ap);
}

gbfd_status cuda_fail(gbfd_ctx *c, cudaError_t e, const char *what)
{
    set_err(c, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
    if (c && (e == cudaErrorIllegalAddress || e == cudaErrorLaunchFailure ||
              e == cudaErrorIllegalInstruction || e == cudaErrorMisalignedAddress ||
              e == cudaErrorHardwareStackError))
        c->broken = true;
    return GBFD_ERR_CUDA;
}

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

int nfields_of(const gbfd_params *p) { return p->entropy_mode ? 5 : 4; }

bool validate(const gbfd_params *p, char *why, size_t n)
{
    if (!p) {
        snprintf(why, n, "params is NULL");
        return false;
    }
    if (p->nx < 8 || p->ny < 8 || p->nz < 8) {
        snprintf(why, n, "grid %dx%dx%d: every extent must be >= 8", p->nx, p->ny, p->nz);
        return false;
    }
    if (p->nx % 4) {
        snprintf(why, n, "nx = %d must be a multiple of 4", p->nx);
        return false;
    }
    if ((long long)p->nx * p->ny * p->nz > (1LL << 33)) {
        snprintf(why, n, "grid too large");
        return false;
    }
    if (p->precision < GBFD_FP64 || p->precision > GBFD_FP32_ACCFF) {
        snprintf(why, n, "unknown precision %d", p->precision);
        return false;
    }
    if (p->precision == GBFD_FP32_ACCFF && p->form != GBFD_55P) {
        snprintf(why, n, "the float-float precision form is built for the 55-point form only");
        return false;
    }
    if (p->form != GBFD_55P && p->form != GBFD_19P) {
        snprintf(why, n, "unknown form %d", p->form);
        return false;
    }
    if (p->bc_z != GBFD_BC_PERIODIC && p->bc_z != GBFD_BC_WALL && p->bc_z != GBFD_BC_EXCHANGE) {
        snprintf(why, n, "bc_z must be GBFD_BC_PERIODIC, GBFD_BC_WALL or GBFD_BC_EXCHANGE");
        return false;
    }
    if (p->bc_z == GBFD_BC_EXCHANGE && p->form != GBFD_55P) {
        snprintf(why, n, "exchanged z halos are built for the 55-point form only");
        return false;
    }
    if (p->entropy_mode != 0 && p->entropy_mode != 1) {
        snprintf(why, n, "entropy_mode must be 0 or 1");
        return false;
    }
    const double v[5] = {p->lx, p->ly, p->lz, p->cs, p->nu};
    for (int i = 0; i < 5; ++i)
        if (!std::isfinite(v[i])) {
            snprintf(why, n, "non-finite box length or physical parameter");
            return false;
        }
    if (p->lx <= 0 || p->ly <= 0 || p->lz <= 0 || p->cs < 0 || p->nu < 0) {
        snprintf(why, n, "box lengths must be > 0, cs and nu >= 0");
        return false;
    }
    return true;
}

struct Plan {
    Layout Ls, Lw, Ld;
    size_t off_state[2], off_w, off_div, off_staging, off_part, off_out, off_err, off_ftab, total;
    int ndiag;
};

Plan make_plan(const gbfd_params *p)
{
    Plan pl;
    const int nf = nfields_of(p);
    const int sb = p->precision == GBFD_FP64 ? 8 : 4;
    const int wb = (p->precision == GBFD_FP64 || p->precision == GBFD_FP32_ACC64_W64) ? 8 : 4;
    // walls in z: ghost planes on the state and the stored divergence (the
    // 2N register is only read at interior points)
    const int gz = p->bc_z != GBFD_BC_PERIODIC ? GZW : 0;
    pl.Ls = make_layout(p->nx, p->ny, p->nz, sb, nf, gz);
    pl.Lw = make_layout(p->nx, p->ny, p->nz, wb, nf);
    pl.Ld = make_layout(p->nx, p->ny, p->nz, sb, 1, gz);
    pl.ndiag = diag_blocks(pl.Ls);
    size_t off = 0;
    for (int i = 0; i < 2; ++i) {
        pl.off_state[i] = off;
        off = align256(off + pl.Ls.bytes);
    }
    pl.off_w = off;
    off = align256(off + pl.Lw.bytes);
    pl.off_div = off;
    if (p->form == GBFD_19P)
        off = align256(off + pl.Ld.bytes);
    pl.off_staging = off;
    off = align256(off + (size_t)nf * p->nx * p->ny * p->nz * 8);
    pl.off_part = off;
    off = align256(off + (size_t)pl.ndiag * 16 * sizeof(double));
    pl.off_out = off;
    off = align256(off + 16 * sizeof(double));
    pl.off_err = off;
    off = align256(off + 256);
    pl.off_ftab = off;  // forcing phase tables, (nx + ny + nz) complex FP64, then FP32
    off = align256(off + (size_t)(p->nx + p->ny + p->nz) * 24);
    pl.total = off;
    return pl;
}

StateBufs bufs(gbfd_ctx *c)
{
    StateBufs b;
    b.in = c->state_region[c->cur] + c->Ls.origin;
    b.out = c->state_region[c->cur ^ 1] + c->Ls.origin;
    b.w = c->w_region + c->Lw.origin;
    b.div = c->div_region ? c->div_region + c->Ld.origin : nullptr;
    b.Ls = c->Ls;
    b.Lw = c->Lw;
    return b;
}

gbfd_status check_ctx(gbfd_ctx *c)
{
    if (!c)
        return GBFD_ERR_INVALID_ARG;
    if (c->broken) {
        set_err(c, "context unusable after an earlier device fault");
        return GBFD_ERR_STATE;
    }
    return GBFD_OK;
}

gbfd_status do_substep(gbfd_ctx *c, int s, double dt);

// The autotuner's timing launch: substep s from the current buffer into the
// spare one, without making the spare one current (the state is unchanged).
gbfd_status probe_substep(gbfd_ctx *c, int s, double dt)
{
    gbfd_status st = do_substep(c, s, dt);
    if (st == GBFD_OK)
        c->cur ^= 1;
    return st;
}

// Autotuner cache: one JSON object, one entry per line,
//   "key": {"cfg": <int>, "ms": <double>},
std::map<std::string, std::pair<int, double>> read_cache(const char *path)
{
    std::map<std::string, std::pair<int, double>> m;
    FILE *f = fopen(path, "r");
    if (!f)
        return m;
    char line[1024];
    while (fgets(line, sizeof line, f)) {
        const char *q0 = strchr(line, '"');
        const char *q1 = q0 ? strchr(q0 + 1, '"') : nullptr;
        if (!q1)
            continue;
        int cfg = 0;
        double ms = 0;
        const char *c = strstr(q1, "\"cfg\":");
        const char *t = strstr(q1, "\"ms\":");
        if (!c || !t || sscanf(c + 6, "%d", &cfg) != 1 || sscanf(t + 5, "%lf", &ms) != 1)
            continue;
        m[std::string(q0 + 1, q1)] = std::make_pair(cfg, ms);
    }
    fclose(f);
    return m;
}

bool write_cache(const char *path, const std::map<std::string, std::pair<int, double>> &m)
{
    std::string tmp = std::string(path) + ".tmp";
    FILE *f = fopen(tmp.c_str(), "w");
    if (!f)
        return false;
    fprintf(f, "{\n");
    size_t i = 0;
    for (const auto &kv : m)
        fprintf(f, "  \"%s\": {\"cfg\": %d, \"ms\": %.6f}%s\n", kv.first.c_str(),
                kv.second.first, kv.second.second, ++i < m.size() ? "," : "");
    fprintf(f, "}\n");
    fclose(f);
    return rename(tmp.c_str(), path) == 0;
}

// The FP32 default's z-chunk length for this grid (S = resident CTAs of the
// default kernel: 32 x 8 tiles, two per SM): 64 planes when that makes at
// least 16 launch waves (512^3: 27 waves, 3% faster than 40 there, the halo
// planes falling from 15% to 9%); else 40 when that still makes at least
// four waves (fewest halo planes, and 7 chunks of a 256 column fill 5.9
// waves where 8 chunks of 32 fill 6.7); else 32 when that fills at least
// half a wave; else 16 when that fills a quarter; else 8, so that small grids
// (64^3: 128 CTAs of 8 planes) keep more SMs busy and each CTA's plane
// pipeline short.  Measured best at 128^3 (32), 256^3 (40) and 512^3 (64).
int fp32_default_cfg(const gbfd_ctx *c)
{
    const long long slots = 2LL * c->sms;
    const long long tiles = (long long)((c->p.nx + 31) / 32) * ((c->p.ny + 7) / 8);
    // positions of 40, 32, 64, 16 and 8 in the tile table's chunk list
    if (tiles * ((c->p.nz + 63) / 64) >= 16 * slots)
        return kDefaultF32 + 2;
    if (tiles * ((c->p.nz + 39) / 40) >= 4 * slots)
        return kDefaultF32;
    if (2 * tiles * ((c->p.nz + 31) / 32) >= slots)
        return kDefaultF32 + 1;
    if (4 * tiles * ((c->p.nz + 15) / 16) >= slots)
        return kDefaultF32 + 3;
    return kDefaultF32 + 4;
}

gbfd_status do_substep(gbfd_ctx *c, int s, double dt)
{
    StateBufs b = bufs(c);
    RKStage st = make_stage(s, dt, c->p.nu);
    st.fault_skip_plane = c->fault_skip;
    st.fo = c->fo;
    int n = 0;
    cudaError_t e = cudaSuccess;
    const bool tiled = c->kernel_path == 0;
    switch (c->p.precision) {
    case GBFD_FP64:
        e = tiled ? launch_substep_tiled<double, double, double>(b, c->c64, st, c->nf, c->p.form,
                                                                 c->tile_cfg, c->dev_error, &c->tmaps,
                                                                 c->stream, &n)
                  : launch_substep_simple<double, double, double>(b, c->c64, st, c->nf, c->p.form,
                                                                  c->stream, &n);
        break;
    case GBFD_FP32:
        e = tiled ? launch_substep_tiled<float, float, float>(
                        b, c->c32, st, c->nf, c->p.form,
                        c->tile_cfg < 0 ? fp32_default_cfg(c) : c->tile_cfg, c->dev_error,
                        &c->tmaps, c->stream, &n)
                  : launch_substep_simple<float, float, float>(b, c->c32, st, c->nf, c->p.form,
                                                               c->stream, &n);
        break;
    case GBFD_FP32_ACC64:
        e = tiled ? launch_substep_tiled<float, float, double>(b, c->c32, st, c->nf, c->p.form,
                                                               c->tile_cfg, c->dev_error, &c->tmaps,
                                                               c->stream, &n)
                  : launch_substep_simple<float, float, double>(b, c->c32, st, c->nf, c->p.form,
                                                                c->stream, &n);
        break;
    case GBFD_FP32_ACCFF:
        e = tiled ? launch_substep_tiled<float, float, ffloat>(b, c->c32, st, c->nf, c->p.form,
                                                               c->tile_cfg < 0 ? fp32_default_cfg(c)
                                                                               : c->tile_cfg,
                                                               c->dev_error, &c->tmaps, c->stream,
                                                               &n)
                  : launch_substep_simple<float, float, ffloat>(b, c->c32, st, c->nf, c->p.form,
                                                                c->stream, &n);
        break;
    default:
        e = tiled ? launch_substep_tiled<float, double, double>(b, c->c32, st, c->nf, c->p.form,
                                                                c->tile_cfg, c->dev_error, &c->tmaps,
                                                                c->stream, &n)
                  : launch_substep_simple<float, double, double>(b, c->c32, st, c->nf, c->p.form,
                                                                 c->stream, &n);
        break;
    }
    c->launches += n;
    if (e != cudaSuccess)
        return cuda_fail(c, e, "substep launch");
    // walls in z: the boundary step (Algorithm 1) on the new state (with
    // exchanged halos the caller fills the ghost planes instead)
    if (c->p.bc_z == GBFD_BC_WALL) {
        n = 0;
        e = launch_fill_ghosts_z(b.out, c->Ls, c->nf, kWallOddMask, c->stream, &n);
        c->launches += n;
        if (e != cudaSuccess)
            return cuda_fail(c, e, "ghost planes");
    }
    c->cur ^= 1;
    return GBFD_OK;
}

}  // namespace

namespace gbfd {
// Record a failure of a context-free entry point; read by gbfd_last_error(NULL).
void set_global_error(const char *msg) { set_err(nullptr, "%s", msg); }

// Current state of an FP32-storage context on a cubic grid (used by the
// correction network and the box filter); false otherwise.
bool ctx_view(gbfd_ctx *c, float **origin, Layout *L, int *nf, cudaStream_t *s)
{
    if (!c || c->broken || c->sbytes != 4 || c->p.nx != c->p.ny || c->p.ny != c->p.nz ||
        c->p.bc_z != GBFD_BC_PERIODIC)
        return false;
    *origin = reinterpret_cast<float *>(c->state_region[c->cur] + c->Ls.origin);
    *L = c->Ls;
    *nf = c->nf;
    *s = c->stream;
    return true;
}
}  // namespace gbfd

extern "C" {

size_t gbfd_workspace_bytes(const gbfd_params *p)
{
    char why[256];
    if (!validate(p, why, sizeof why))
        return 0;
    return make_plan(p).total;
}

gbfd_status gbfd_init(const gbfd_params *p, void *workspace, size_t workspace_bytes, void *stream,
                      gbfd_ctx **out)
{
    char why[256];
    if (!out) {
        set_err(nullptr, "out is NULL");
        return GBFD_ERR_INVALID_ARG;
    }
    *out = nullptr;
    if (!validate(p, why, sizeof why)) {
        set_err(nullptr, "%s", why);
        return GBFD_ERR_INVALID_ARG;
    }
    Plan pl = make_plan(p);
    if (!workspace || ((uintptr_t)workspace & 255)) {
        set_err(nullptr, "workspace must be a non-NULL, 256-byte aligned device pointer");
        return GBFD_ERR_WORKSPACE;
    }
    if (workspace_bytes < pl.total) {
        set_err(nullptr, "workspace has %zu bytes, %zu needed", workspace_bytes, pl.total);
        return GBFD_ERR_WORKSPACE;
    }
    cudaPointerAttributes attr;
    cudaError_t e = cudaPointerGetAttributes(&attr, workspace);
    if (e != cudaSuccess || attr.type != cudaMemoryTypeDevice) {
        cudaGetLastError();
        set_err(nullptr, "workspace is not device memory");
        return GBFD_ERR_WORKSPACE;
    }
    gbfd_ctx *c = new (std::nothrow) gbfd_ctx();
    if (!c) {
        set_err(nullptr, "out of host memory");
        return GBFD_ERR_INVALID_ARG;
    }
    c->p = *p;
    c->nf = nfields_of(p);
    c->sbytes = pl.Ls.w;
    c->wbytes = pl.Lw.w;
    c->stream = (cudaStream_t)stream;
    c->ws = (char *)workspace;
    c->ws_bytes = workspace_bytes;
    c->Ls = pl.Ls;
    c->Lw = pl.Lw;
    c->Ld = pl.Ld;
    c->state_region[0] = c->ws + pl.off_state[0];
    c->state_region[1] = c->ws + pl.off_state[1];
    c->w_region = c->ws + pl.off_w;
    c->div_region = p->form == GBFD_19P ? c->ws + pl.off_div : nullptr;
    c->staging = c->ws + pl.off_staging;
    c->diag_part = (double *)(c->ws + pl.off_part);
    c->diag_out = (double *)(c->ws + pl.off_out);
    c->dev_error = (int *)(c->ws + pl.off_err);
    c->ftab = (double2 *)(c->ws + pl.off_ftab);
    memset(&c->fo, 0, sizeof c->fo);
    c->ndiag = pl.ndiag;
    c->cur = 0;
    c->launches = 0;
    c->kernel_path = 0;
    c->tile_cfg = -1;
    {
        // the device current at init is the context's device
        int dev = 0;
        c->sms = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            c->sms <= 0) {
            (void)cudaGetLastError();
            c->sms = 152;
        }
    }
    c->fault_skip = -1;
    c->host_path = 0;
    c->host_async = 0;
    memset(&c->tmaps, 0, sizeof c->tmaps);
    c->broken = false;
    const double hx = p->lx / p->nx, hy = p->ly / p->ny;
    const double hz = p->bc_z == GBFD_BC_WALL ? p->lz / (p->nz - 1) : p->lz / p->nz;
    c->h[0] = hx;
    c->h[1] = hy;
    c->h[2] = hz;
    c->c64 = make_coef<double>(hx, hy, hz, p->cs, p->nu);
    c->c32 = make_coef<float>(hx, hy, hz, p->cs, p->nu);
    c->err[0] = 0;
    // zero state, ghosts, padding and the error word once
    e = cudaMemsetAsync(c->ws, 0, pl.total, c->stream);
    if (e != cudaSuccess) {
        cuda_fail(nullptr, e, "workspace clear");
        delete c;
        return GBFD_ERR_CUDA;
    }
    *out = c;
    return GBFD_OK;
}

gbfd_status gbfd_destroy(gbfd_ctx *ctx)
{
    delete ctx;
    return GBFD_OK;
}

gbfd_status gbfd_set_option(gbfd_ctx *ctx, int key, int64_t value)
{
    gbfd_status s = check_ctx(ctx);
    if (s != GBFD_OK)
        return s;
    switch (key) {
    case GBFD_OPT_KERNEL_PATH:
        if (value != 0 && value != 1)
            break;
        ctx->kernel_path = (int)value;
        return GBFD_OK;
    case GBFD_OPT_HOST_PATH:
        if (value != 0 && value != 1)
            break;
        ctx->host_path = (int)value;
        return GBFD_OK;
    case GBFD_OPT_HOST_ASYNC:
        if (value != 0 && value != 1)
            break;
        ctx->host_async = (int)value;
        return GBFD_OK;
    case GBFD_OPT_FAULT_SKIP_COPY:
        if (value < -1 || value > 1000000)
            break;
        ctx->fault_skip = (int)value;
        return GBFD_OK;
    case GBFD_OPT_TILE_CONFIG:
        if (value < -1 || value >= tiled_config_count(ctx->sbytes))
            break;
        ctx->tile_cfg = (int)value;
        return GBFD_OK;
    default:
        break;
    }
    set_err(ctx, "option %d: value %lld rejected", key, (long long)value);
    return GBFD_ERR_INVALID_ARG;
}

gbfd_status gbfd_set_state(gbfd_ctx *ctx, const void *src, int src_on_device, int src_is_fp64)
{
    gbfd_status s = check_ctx(ctx);
    if (s != GBFD_OK)
        return s;
    if (!src) {
        set_err(ctx, "src is NULL");
        return GBFD_ERR_INVALID_ARG;
    }
    const size_t n = (size_t)ctx->nf * ctx->p.nx * ctx->p.ny * ctx->p.nz;
    const size_t bytes = n * (src_is_fp64 ? 8 : 4);
    const void *from = src;
    const void *mapped = (!src_on_device && ctx->host_path == 0) ? mapped_host(src) : nullptr;
    if (mapped) {
        from = mapped;
    } else if (!src_on_device) {
        cudaError_t e =
            cudaMemcpyAsync(ctx->staging, src, bytes, cudaMemcpyHostToDevice, ctx->stream);
        if (e != cudaSuccess)
            return cuda_fail(ctx, e, "set_state copy");
        from = ctx->staging;
    }
    int nl = 0;
    cudaError_t e = launch_scatter(from, src_is_fp64, ctx->state_region[ctx->cur] + ctx->Ls.origin,
                                   ctx->Ls, ctx->nf, ctx->stream, &nl);
    ctx->launches += nl;
    if (e != cudaSuccess)
        return cuda_fail(ctx, e, "set_state scatter");
    if (ctx->p.bc_z == GBFD_BC_WALL) {
        nl = 0;
        e = launch_fill_ghosts_z(ctx->state_region[ctx->cur] + ctx->Ls.origin, ctx->Ls, ctx->nf,
                                 kWallOddMask, ctx->stream, &nl);
        ctx->launches += nl;
        if (e != cudaSuccess)
            return cuda_fail(ctx, e, "set_state ghost planes");
    }
    return GBFD_OK;
}

gbfd_status gbfd_get_state(gbfd_ctx *ctx, void *dst, int dst_on_device, int dst_is_fp64)
{
    gbfd_status s = check_ctx(ctx);
    if (s != GBFD_OK)
        return s;
    if (!dst) {
        set_err(ctx, "dst is NULL");
        return GBFD_ERR_INVALID_ARG;
    }
    const size_t n = (size_t)ctx->nf * ctx->p.nx * ctx->p.ny * ctx->p.nz;
    const size_t bytes = n * (dst_is_fp64 ? 8 : 4);
    void *mapped = (!dst_on_device && ctx->host_path == 0) ? (void *)mapped_host(dst) : nullptr;
    void *to = dst_on_device ? dst : (mapped ? mapped : (void *)ctx->staging);
    int nl = 0;
    cudaError_t e = launch_gather(ctx->state_region[ctx->cur] + ctx->Ls.origin, ctx->Ls, to,
                                  dst_is_fp64, ctx->nf, ctx->stream, &nl);
    ctx->launches += nl;
    if (e != cudaSuccess)
        return cuda_fail(ctx, e, "get_state gather");
    if (!dst_on_device) {
        if (!mapped) {
            e = cudaMemcpyAsync(dst, ctx->staging, bytes, cudaMemcpyDeviceToHost, ctx->stream);
            if (e != cudaSuccess)
                return cuda_fail(ctx, e, "get_state copy");
        }
        if (ctx->host_async)
            return GBFD_OK;  // complete once the stream reaches this point
        // the stream is waited for anyway: report a bounded wait that gave up
        // in the steps that produced this state, as gbfd_sync does
        return gbfd_sync(ctx);
    }
    return GBFD_OK;
}

gbfd_status gbfd_substep(gbfd_ctx *ctx, int s, double dt)
{
    gbfd_status st = check_ctx(ctx);
    if (st != GBFD_OK)
        return st;
    if (s < 0 || s > 2 || !(dt > 0) || !std::isfinite(dt)) {
        set_err(ctx, "substep %d / dt %g rejected", s, dt);
        return GBFD_ERR_INVALID_ARG;
    }
    return do_substep(ctx, s, dt);
}

gbfd_status gbfd_rk3_step(gbfd_ctx *ctx, double dt, int nsteps)
{
    gbfd_status st = check_ctx(ctx);
    if (st != GBFD_OK)
        return st;
    if (nsteps < 0 || !(dt > 0) || !std::isfinite(dt)) {
        set_err(ctx, "rk3_step: dt %g / nsteps %d rejected", dt, nsteps);
        return GBFD_ERR_INVALID_ARG;
    }
    for (int n = 0; n < nsteps; ++n)
        for (int s = 0; s < 3; ++s) {
            st = do_substep(ctx, s, dt);
            if (st != GBFD_OK)
                return st;
        }
    return GBFD_OK;
}

gbfd_status gbfd_rk3_step_forced(gbfd_ctx *ctx, double dt, int nsteps, double f0, const int *k,
                                 const double *phi, const double *e)
{
    gbfd_status st = check_ctx(ctx);
    if (st != GBFD_OK)
        return st;
    if (nsteps < 0 || !(dt > 0) || !std::isfinite(dt) || !std::isfinite(f0)) {
        set_err(ctx, "rk3_step_forced: dt %g / nsteps %d / f0 %g rejected", dt, nsteps, f0);
        return GBFD_ERR_INVALID_ARG;
    }
    if (nsteps > 0 && (!k || !phi || !e)) {
        set_err(ctx, "rk3_step_forced: k, phi and e must not be NULL");
        return GBFD_ERR_INVALID_ARG;
    }
    if (ctx->p.bc_z != GBFD_BC_PERIODIC) {
        set_err(ctx, "rk3_step_forced: the forcing of Sect. 6 needs a periodic box");
        return GBFD_ERR_UNSUPPORTED;
    }
    const double two_pi = 6.283185307179586476925286766559;
    const double L[3] = {ctx->p.lx, ctx->p.ly, ctx->p.lz};
    for (int n = 0; n < nsteps; ++n) {
        // Eq. 21: N = f0 c_s sqrt(|k| c_s / dt), f_k = (k x e) / sqrt(|k|^2 - (k.e)^2),
        // with the physical wave vector k_i = 2 pi kint_i / L_i
        const int *ki = k + 3 * n;
        const double *ei = e + 3 * n;
        double kp[3], kk = 0.0, ke = 0.0;
        for (int a = 0; a < 3; ++a) {
            kp[a] = two_pi * (double)ki[a] / L[a];
            kk += kp[a] * kp[a];
            ke += kp[a] * ei[a];
        }
        const double den2 = kk - ke * ke;
        if (!(kk > 0.0) || !(den2 > 1e-24 * kk) || !std::isfinite(phi[n])) {
            set_err(ctx, "rk3_step_forced: step %d: k zero or parallel to e, or phi not finite", n);
            return GBFD_ERR_INVALID_ARG;
        }
        const double N = f0 * ctx->p.cs * std::sqrt(std::sqrt(kk) * ctx->p.cs / dt);
        const double kxe[3] = {kp[1] * ei[2] - kp[2] * ei[1], kp[2] * ei[0] - kp[0] * ei[2],
                               kp[0] * ei[1] - kp[1] * ei[0]};
        const double den = std::sqrt(den2);
        Forcing fo;
        fo.on = 1;
        for (int a = 0; a < 3; ++a) {
            fo.amp[a] = N * kxe[a] / den;
            fo.amp32[a] = (float)fo.amp[a];
        }
        fo.tx = ctx->ftab;
        fo.ty = ctx->ftab + ctx->p.nx;
        fo.tz = ctx->ftab + ctx->p.nx + ctx->p.ny;
        float2 *t32 = reinterpret_cast<float2 *>(ctx->ftab + ctx->p.nx + ctx->p.ny + ctx->p.nz);
        fo.tx32 = t32;
        fo.ty32 = t32 + ctx->p.nx;
        fo.tz32 = t32 + ctx->p.nx + ctx->p.ny;
        int nl = 0;
        cudaError_t ce = launch_forcing_tables(ki[0], ki[1], ki[2], phi[n], ctx->p.nx, ctx->p.ny,
                                               ctx->p.nz, ctx->ftab, t32, ctx->stream, &nl);
        ctx->launches += nl;
        if (ce != cudaSuccess)
            return cuda_fail(ctx, ce, "forcing tables");
        ctx->fo = fo;
        for (int s = 0; s < 3; ++s) {
            st = do_substep(ctx, s, dt);
            if (st != GBFD_OK)
                break;
        }
        memset(&ctx->fo, 0, sizeof ctx->fo);
        if (st != GBFD_OK)
            return st;
    }
    return GBFD_OK;
}

size_t gbfd_halo_bytes(const gbfd_ctx *ctx)
{
    if (!ctx || ctx->p.bc_z != GBFD_BC_EXCHANGE)
        return 0;
    return (size_t)ctx->nf * GZW * ctx->Ls.plane * ctx->Ls.w;
}

// One side's halo message: the GZW interior planes next to that side, whole
// padded planes of every field, [field][plane][Y][X].
static gbfd_status halo_copy(gbfd_ctx *ctx, int side, void *buf, bool pack)
{
    gbfd_status st = check_ctx(ctx);
    if (st != GBFD_OK)
        return st;
    if (ctx->p.bc_z != GBFD_BC_EXCHANGE) {
        set_err(ctx, "halo exchange needs a context created with bc_z = GBFD_BC_EXCHANGE");
        return GBFD_ERR_UNSUPPORTED;
    }
    if ((side != 0 && side != 1) || !buf) {
        set_err(ctx, "halo: side must be 0 (low z) or 1 (high z) and the buffer non-NULL");
        return GBFD_ERR_INVALID_ARG;
    }
    const Layout &L = ctx->Ls;
    char *origin = ctx->state_region[ctx->cur] + L.origin;
    // pack: interior planes 0..2 (side 0) or nz-3..nz-1 (side 1); unpack:
    // ghost planes -3..-1 (side 0) or nz..nz+2 (side 1), in increasing z
    const long long z0 = pack ? (side ? L.nz - GZW : 0) : (side ? L.nz : -GZW);
    char *field0 = origin + z0 * L.plane * L.w;
    const size_t width = (size_t)GZW * L.plane * L.w, fp = (size_t)L.fpitch * L.w;
    cudaError_t e = pack ? cudaMemcpy2DAsync(buf, width, field0, fp, width, ctx->nf,
                                             cudaMemcpyDeviceToDevice, ctx->stream)
                         : cudaMemcpy2DAsync(field0, fp, buf, width, width, ctx->nf,
                                             cudaMemcpyDeviceToDevice, ctx->stream);
    if (e != cudaSuccess)
        return cuda_fail(ctx, e, pack ? "halo pack" : "halo unpack");
    return GBFD_OK;
}

gbfd_status gbfd_halo_pack(gbfd_ctx *ctx, int side, void *dst)
{
    return halo_copy(ctx, side, dst, true);
}

gbfd_status gbfd_halo_unpack(gbfd_ctx *ctx, int side, const void *src)
{
    return halo_copy(ctx, side, const_cast<void *>(src), false);
}

gbfd_status gbfd_sync(gbfd_ctx *ctx)
{
    gbfd_status st = check_ctx(ctx);
    if (st != GBFD_OK)
        return st;
    int herr = 0;
    cudaError_t e = cudaMemcpyAsync(&herr, ctx->dev_error, sizeof(int), cudaMemcpyDeviceToHost,
                                    ctx->stream);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess)
        return cuda_fail(ctx, e, "sync");
    if (herr) {
        set_err(ctx, "device-side bounded wait gave up (code %d)", herr);
        cudaMemsetAsync(ctx->dev_error, 0, sizeof(int), ctx->stream);
        return GBFD_ERR_TIMEOUT;
    }
    return GBFD_OK;
}

gbfd_status gbfd_diagnostics(gbfd_ctx *ctx, gbfd_diag *out)
{
    gbfd_status st = check_ctx(ctx);
    if (st != GBFD_OK)
        return st;
    if (!out) {
        set_err(ctx, "out is NULL");
        return GBFD_ERR_INVALID_ARG;
    }
    const double dv = ctx->h[0] * ctx->h[1] * ctx->h[2];
    int nl = 0;
    cudaError_t e = launch_diagnostics(ctx->state_region[ctx->cur] + ctx->Ls.origin, ctx->Ls,
                                       ctx->nf, dv, ctx->diag_part, ctx->ndiag, ctx->diag_out,
                                       ctx->stream, &nl);
    ctx->launches += nl;
    if (e != cudaSuccess)
        return cuda_fail(ctx, e, "diagnostics launch");
    double h[16];
    e = cudaMemcpyAsync(h, ctx->diag_out, sizeof h, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess)
        return cuda_fail(ctx, e, "diagnostics read");
    out->mass = h[0];
    out->ekin = h[1];
    out->umax = h[2];
    out->urms = h[3];
    for (int f = 0; f < 5; ++f) {
        out->rms[f] = h[4 + f];
        out->maxabs[f] = h[9 + f];
    }
    out->nonfinite = h[14] != 0.0;
    out->nfields = ctx->nf;
    return GBFD_OK;
}

gbfd_status gbfd_cfl_dt(gbfd_ctx *ctx, double cfl, double cnu, double *dt_out)
{
    if (!dt_out || !(cfl > 0) || !(cnu > 0)) {
        if (ctx)
            set_err(ctx, "cfl_dt: bad arguments");
        return GBFD_ERR_INVALID_ARG;
    }
    gbfd_diag d;
    gbfd_status st = gbfd_diagnostics(ctx, &d);
    if (st != GBFD_OK)
        return st;
    const double *h = ctx->h;
    double dmin = h[0] < h[1] ? h[0] : h[1];
    dmin = dmin < h[2] ? dmin : h[2];
    double dt = cfl * dmin / (d.umax + ctx->p.cs);
    if (ctx->p.nu > 0) {
        const double dtn = cnu * dmin * dmin / ctx->p.nu;
        dt = dtn < dt ? dtn : dt;
    }
    *dt_out = dt;
    return GBFD_OK;
}

gbfd_status gbfd_autotune(gbfd_ctx *ctx, int reps, const char *cache_path, int *best_cfg,
                          double *best_ms)
{
    gbfd_status st = check_ctx(ctx);
    if (st != GBFD_OK)
        return st;
    if (reps < 1) {
        set_err(ctx, "autotune: reps must be >= 1");
        return GBFD_ERR_INVALID_ARG;
    }
    int dev = 0;
    cudaDeviceProp prop;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess)
        e = cudaGetDeviceProperties(&prop, dev);
    if (e != cudaSuccess)
        return cuda_fail(ctx, e, "autotune device query");
    char key[512];
    snprintf(key, sizeof key, "%s|%dx%dx%d|precision%d|form%d|fields%d", prop.name, ctx->p.nx,
             ctx->p.ny, ctx->p.nz, ctx->p.precision, ctx->p.form, ctx->nf);
    for (char *p = key; *p; ++p)
        if (*p == '"' || *p == '\\')
            *p = '_';
    // the precision forms compile three kernels (packed two-point with integer
    // or hardware conversions, one-point): tune those and their chunk lengths
    const bool acc = ctx->p.precision == GBFD_FP32_ACC64 || ctx->p.precision == GBFD_FP32_ACC64_W64;
    // the float-float form runs one kernel: tune its chunk length only
    const bool ff = ctx->p.precision == GBFD_FP32_ACCFF;
    const int count = acc ? 3 * kZcChoices : (ff ? kZcChoices : tiled_config_count(ctx->sbytes));
    std::map<std::string, std::pair<int, double>> cache;
    if (cache_path) {
        cache = read_cache(cache_path);
        auto it = cache.find(key);
        if (it != cache.end() && it->second.first >= 0 && it->second.first < count) {
            ctx->tile_cfg = it->second.first;
            ctx->kernel_path = 0;
            if (best_cfg)
                *best_cfg = ctx->tile_cfg;
            if (best_ms)
                *best_ms = 0.0;
            return GBFD_OK;
        }
    }
    cudaEvent_t e0, e1;
    if ((e = cudaEventCreate(&e0)) != cudaSuccess)
        return cuda_fail(ctx, e, "autotune events");
    if ((e = cudaEventCreate(&e1)) != cudaSuccess) {
        cudaEventDestroy(e0);
        return cuda_fail(ctx, e, "autotune events");
    }
    const int saved_path = ctx->kernel_path, saved_cfg = ctx->tile_cfg;
    ctx->kernel_path = 0;
    int best = -1;
    double bms = 1e300;
    for (int cfg = 0; cfg < count && st == GBFD_OK; ++cfg) {
        ctx->tile_cfg = cfg;
        for (int r = 0; r <= reps && st == GBFD_OK; ++r) {
            if (r == 1 && (e = cudaEventRecord(e0, ctx->stream)) != cudaSuccess)
                break;
            for (int sub = 0; sub < 3 && st == GBFD_OK; ++sub)
                st = probe_substep(ctx, sub, 1e-6);
        }
        if (st != GBFD_OK || e != cudaSuccess)
            break;
        float ms = 0;
        if ((e = cudaEventRecord(e1, ctx->stream)) != cudaSuccess ||
            (e = cudaEventSynchronize(e1)) != cudaSuccess ||
            (e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess)
            break;
        if (ms / reps < bms) {
            bms = ms / reps;
            best = cfg;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st == GBFD_OK && e != cudaSuccess)
        st = cuda_fail(ctx, e, "autotune timing");
    if (st != GBFD_OK || best < 0) {
        ctx->kernel_path = saved_path;
        ctx->tile_cfg = saved_cfg;
        return st != GBFD_OK ? st : GBFD_ERR_CUDA;
    }
    ctx->tile_cfg = best;
    if (cache_path) {
        cache[key] = std::make_pair(best, bms);
        if (!write_cache(cache_path, cache)) {
            set_err(ctx, "autotune: cannot write cache %s", cache_path);
            return GBFD_ERR_INVALID_ARG;
        }
    }
    if (best_cfg)
        *best_cfg = best;
    if (best_ms)
        *best_ms = bms;
    return GBFD_OK;
}

int64_t gbfd_launch_count(const gbfd_ctx *ctx) { return ctx ? ctx->launches : 0; }

const char *gbfd_last_error(const gbfd_ctx *ctx) { return ctx ? ctx->err : g_init_err; }

const char *gbfd_status_string(gbfd_status s)
{
    switch (s) {
    case GBFD_OK:
        return "GBFD_OK";
    case GBFD_ERR_INVALID_ARG:
        return "GBFD_ERR_INVALID_ARG";
    case GBFD_ERR_WORKSPACE:
        return "GBFD_ERR_WORKSPACE";
    case GBFD_ERR_CUDA:
        return "GBFD_ERR_CUDA";
    case GBFD_ERR_TIMEOUT:
        return "GBFD_ERR_TIMEOUT";
    case GBFD_ERR_UNSUPPORTED:
        return "GBFD_ERR_UNSUPPORTED";
    case GBFD_ERR_STATE:
        return "GBFD_ERR_STATE";
    }
    return "unknown";
}

}  // extern "C"
