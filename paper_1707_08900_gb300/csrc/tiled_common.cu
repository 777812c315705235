// Tile tables of the tiled substep kernels and TMA descriptor encoding.
#include <cudaTypedefs.h>

#include <cstring>

#include "tiled.cuh"

namespace gbfd {

namespace {

// (tx, ty, ns) variants compiled per storage width; each is offered with
// several z-chunk lengths.
const TileConfig kVariants4[] = {{32, 8, 0, 9, 1},
                                 {32, 8, 0, 8, 2, 2},
                                 {32, 8, 0, 8, 2, 2, 0, 1},
                                 {32, 8, 0, 8, 2, 1, 0, 1},
                                 {32, 8, 0, 8, 2, 2, 1, 1},
                                 {32, 8, 0, 8, 2, 2, 1, 1},
                                 {32, 8, 0, 8, 2, 2, 1, 1}};
const TileConfig kVariants8[] = {{32, 4, 0, 8, 1},       {16, 8, 0, 8, 1},
                                 {32, 4, 0, 6, 2, 1},    {32, 4, 0, 5, 2, 2},
                                 {32, 8, 0, 5, 2, 1},    {16, 8, 0, 5, 1, 0, 1, 1}};
const int kZc[kZcChoices] = {40, 32, 64, 16, 8};
constexpr int kNz = kZcChoices;

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

}  // namespace

int tiled_config_count(int sbytes)
{
    return (sbytes == 8 ? (int)(sizeof kVariants8 / sizeof kVariants8[0])
                        : (int)(sizeof kVariants4 / sizeof kVariants4[0])) *
           kNz;
}

TileConfig tiled_config(int sbytes, int i)
{
    TileConfig t = sbytes == 8 ? kVariants8[i / kNz] : kVariants4[i / kNz];
    t.zc = kZc[i % kNz];
    return t;
}

namespace {

bool encode_tmap(TmapCache *cache, const void *origin, const Layout &L, int nf, int bx, int by,
                 int key, CUtensorMap **out)
{
    for (int i = 0; i < TmapCache::kEntries; ++i) {
        TmapCache::Entry &e = cache->e[i];
        if (e.valid && e.base == origin && e.cfg == key && e.nf == nf) {
            *out = &e.map;
            return true;
        }
    }
    PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
    if (!fn)
        return false;
    TmapCache::Entry &e = cache->e[cache->next];
    cache->next = (cache->next + 1) % TmapCache::kEntries;
    memset(&e, 0, sizeof e);
    // with walls in z the map covers the ghost planes too: it starts at
    // ghost plane -gz (kernels add gz to the plane index)
    const cuuint64_t dims[4] = {(cuuint64_t)(L.nx + 2 * GX), (cuuint64_t)L.rows,
                                (cuuint64_t)(L.nz + 2 * L.gz), (cuuint64_t)nf};
    const char *base = static_cast<const char *>(origin) - (long long)L.gz * L.plane * L.w;
    const cuuint64_t strides[3] = {(cuuint64_t)(L.P * L.w), (cuuint64_t)(L.plane * L.w),
                                   (cuuint64_t)(L.fpitch * L.w)};
    const cuuint32_t box[4] = {(cuuint32_t)bx, (cuuint32_t)by, 1u, (cuuint32_t)nf};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    CUresult r = fn(&e.map, L.w == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                    4, const_cast<char *>(base), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS)
        return false;
    e.base = origin;
    e.cfg = key;
    e.nf = nf;
    e.valid = true;
    *out = &e.map;
    return true;
}

}  // namespace

bool get_state_tmap(TmapCache *cache, const void *origin, const Layout &L, int nf, int tx, int ty,
                    int cfg_key, CUtensorMap **out)
{
    return encode_tmap(cache, origin, L, nf, tx + 2 * GX, ty + 2 * GY, cfg_key, out);
}

bool get_tile_tmap(TmapCache *cache, const void *origin, const Layout &L, int nf, int tx, int ty,
                   int cfg_key, CUtensorMap **out)
{
    return encode_tmap(cache, origin, L, nf, tx, ty, 1000 + cfg_key, out);
}

}  // namespace gbfd
