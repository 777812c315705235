// Internal definitions shared by the libgbfd translation units: the padded
// field layout in HBM, the stencil coefficient tables, the Williamson RK3
// coefficients and the per-point right-hand side of Eqs. 1-3.
#pragma once

#include <cstdint>

#include <cuda_runtime.h>
#include <stdint.h>

namespace gbfd {

// ---------------------------------------------------------------------------
// Padded field layout.
//
// Each field is stored as [z][Y][X] with ghost columns/rows in x and y only:
// interior point (x, y, z) lives at X = x + GX, Y = y + GY.  The ghosts hold
// periodic copies (X in [0, GX) is x = nx-GX.., X in [nx+GX, nx+2GX) is
// x = 0..GX-1; same in y with GY) so that a tile plus its 3-cell halo is one
// rectangular, in-bounds box for TMA.  z needs no ghosts: a plane is fetched
// by its wrapped index.  The row pitch P is a multiple of 128 bytes and the
// origin is offset so that every interior row starts 128-byte aligned
// (whole-sector warp accesses).  GX = 4 (not 3) keeps the TMA box origin
// X = x0 16-byte aligned.
//
// With walls in z (the ghost-zone boundary variant) each field also holds
// gz = 3 ghost planes below and above its nz interior planes: interior plane
// z sits at plane index z + gz of the field, the origin points at interior
// plane 0, so element offsets of interior points are unchanged, and ghost
// planes are z = -3..-1 and nz..nz+2.  A ghost-fill kernel writes them (the
// parity mirror of the interior about the wall points) after every substep.
// ---------------------------------------------------------------------------
constexpr int GX = 4;
constexpr int GY = 3;
constexpr int R = 3;  // stencil radius (sixth order, n = 2R)

struct Layout {
    int nx, ny, nz;
    int w;              // bytes per value
    long long P;        // row pitch, elements
    long long rows;     // rows per plane, ny + 2 GY
    long long plane;    // P * rows
    long long fpitch;   // elements between consecutive fields
    long long origin;   // byte offset of element (f=0,z=0,Y=0,X=0) in the region
    long long bytes;    // region bytes for `nf` fields
    int gz;             // ghost planes below and above in z: 0 (periodic z) or
                        // GZW (walls in z)
};

constexpr int GZW = 3;  // ghost planes per side with walls in z

inline Layout make_layout(int nx, int ny, int nz, int w, int nf, int gz = 0)
{
    Layout L;
    L.nx = nx;
    L.ny = ny;
    L.nz = nz;
    L.w = w;
    L.gz = gz;
    const long long q = 128 / w;  // elements per 128 bytes
    L.P = ((nx + 2 * GX + q - 1) / q) * q;
    L.rows = ny + 2 * GY;
    L.plane = L.P * L.rows;
    L.fpitch = L.plane * (nz + 2 * gz);  // P*w is a multiple of 128, so is this
    L.origin = 128 - GX * w + (long long)gz * L.plane * w;
    L.bytes = 128 + (long long)nf * L.fpitch * w;
    return L;
}

// Index of the plane holding local z (which may lie in [-3, nz + 3) for a
// stencil arm): the wrapped index for periodic z, the plane itself (ghost
// planes included) with walls.  TMA maps of a walled layout start at ghost
// plane -gz, so their z coordinate is zplane + gz.
__host__ __device__ __forceinline__ int zplane(const Layout &L, int z)
{
    if (L.gz)
        return z;
    return z < 0 ? z + L.nz : (z >= L.nz ? z - L.nz : z);
}

// Element index of interior point (x, y, z) of field f relative to origin.
__host__ __device__ inline long long lidx(const Layout &L, int f, int z, int y, int x)
{
    return (long long)f * L.fpitch + (long long)z * L.plane + (long long)(y + GY) * L.P + (x + GX);
}

// ---------------------------------------------------------------------------
// Stencil coefficients (Eqs. 6-8) with the grid spacing folded in.
//   D1 f = sum_k d1[a][k-1] (f_{+k} - f_{-k})                      (Eq. 6)
//   D2 f = d2c[a] f_0 + sum_k d2[a][k-1] (f_{+k} + f_{-k})         (Eq. 7)
//   Dab f = sum_k mx[p][k-1] (f_{+k,+k} - f_{-k,+k} + f_{-k,-k} - f_{+k,-k})
//                                                                  (Eq. 8)
// pair p: 0 = (x,y), 1 = (x,z), 2 = (y,z).
// ---------------------------------------------------------------------------
template <class T>
struct Coef {
    T d1[3][3];
    T d2c[3];
    T d2[3][3];
    T mx[3][3];
    T cs2;     // c_s^2
    T nu;      // nu
    T nu3;     // nu / 3
    T nu2;     // 2 nu
    T nu23;    // (2/3) nu
    // accessors shared with CubicCoef (axis a, pair p, arm k = 1..3)
    __host__ __device__ __forceinline__ T D1(int a, int k) const { return d1[a][k - 1]; }
    __host__ __device__ __forceinline__ T D2c(int a) const { return d2c[a]; }
    __host__ __device__ __forceinline__ T D2(int a, int k) const { return d2[a][k - 1]; }
    __host__ __device__ __forceinline__ T MX(int p, int k) const { return mx[p][k - 1]; }
};

// Coefficients of a box with the same spacing h on every axis: one set of
// stencil weights serves all axes (10 values plus 4 physics scalars), small
// enough to live in registers when it changes from box to box.
template <class T>
struct CubicCoef {
    T d1[3], d2c, d2[3], mx[3];
    T cs2, nu, nu3, nu23;
    __host__ __device__ __forceinline__ T D1(int, int k) const { return d1[k - 1]; }
    __host__ __device__ __forceinline__ T D2c(int) const { return d2c; }
    __host__ __device__ __forceinline__ T D2(int, int k) const { return d2[k - 1]; }
    __host__ __device__ __forceinline__ T MX(int, int k) const { return mx[k - 1]; }
};

template <class T>
inline Coef<T> make_coef(double hx, double hy, double hz, double cs, double nu)
{
    Coef<T> c;
    const double h[3] = {hx, hy, hz};
    const double d1w[3] = {45.0, -9.0, 1.0};
    const double d2w[3] = {270.0, -27.0, 2.0};
    const double mxw[3] = {270.0, -27.0, 2.0};
    for (int a = 0; a < 3; ++a) {
        for (int k = 0; k < 3; ++k) {
            c.d1[a][k] = (T)(d1w[k] / (60.0 * h[a]));
            c.d2[a][k] = (T)(d2w[k] / (180.0 * h[a] * h[a]));
        }
        c.d2c[a] = (T)(-490.0 / (180.0 * h[a] * h[a]));
    }
    const double hp[3][2] = {{hx, hy}, {hx, hz}, {hy, hz}};
    for (int p = 0; p < 3; ++p)
        for (int k = 0; k < 3; ++k)
            c.mx[p][k] = (T)(mxw[k] / (720.0 * hp[p][0] * hp[p][1]));
    c.cs2 = (T)(cs * cs);
    c.nu = (T)nu;
    c.nu3 = (T)(nu / 3.0);
    c.nu2 = (T)(2.0 * nu);
    c.nu23 = (T)(2.0 * nu / 3.0);
    return c;
}

// True when the weights are the same on every axis (equal grid spacing);
// cubic_of then carries exactly the same values in the isotropic form.
template <class T>
inline bool coef_is_cubic(const Coef<T> &c)
{
    bool iso = c.d2c[1] == c.d2c[0] && c.d2c[2] == c.d2c[0];
    for (int k = 0; k < 3; ++k)
        iso = iso && c.d1[1][k] == c.d1[0][k] && c.d1[2][k] == c.d1[0][k] &&
              c.d2[1][k] == c.d2[0][k] && c.d2[2][k] == c.d2[0][k] &&
              c.mx[1][k] == c.mx[0][k] && c.mx[2][k] == c.mx[0][k];
    return iso;
}

template <class T>
inline CubicCoef<T> cubic_of(const Coef<T> &c)
{
    CubicCoef<T> q;
    for (int k = 0; k < 3; ++k) {
        q.d1[k] = c.d1[0][k];
        q.d2[k] = c.d2[0][k];
        q.mx[k] = c.mx[0][k];
    }
    q.d2c = c.d2c[0];
    q.cs2 = c.cs2;
    q.nu = c.nu;
    q.nu3 = c.nu3;
    q.nu23 = c.nu23;
    return q;
}

template <class T>
inline CubicCoef<T> make_cubic_coef(double h, double cs, double nu)
{
    Coef<T> c = make_coef<T>(h, h, h, cs, nu);
    CubicCoef<T> q;
    for (int k = 0; k < 3; ++k) {
        q.d1[k] = c.d1[0][k];
        q.d2[k] = c.d2[0][k];
        q.mx[k] = c.mx[0][k];
    }
    q.d2c = c.d2c[0];
    q.cs2 = c.cs2;
    q.nu = c.nu;
    q.nu3 = c.nu3;
    q.nu23 = c.nu23;
    return q;
}

// Williamson (1980) 2N-storage RK3: the paper's Eq. 10 leaves alpha, beta to
// the chosen scheme and fixes alpha_1 = 0.
constexpr double RK3_ALPHA[3] = {0.0, -5.0 / 9.0, -153.0 / 128.0};
constexpr double RK3_BETA[3] = {1.0 / 3.0, 15.0 / 16.0, 8.0 / 15.0};

// ---------------------------------------------------------------------------
// Right-hand side of Eqs. 1-3 (f = 0) at one point from its derivatives.
// gu[i][j] = d_j u_i.  lap[i] = sum_j D2_j u_i.  gd[i] = d_i(div u), the
// grad-div term (left 0 by the 19-point first pass, which adds it in pass 2).
// ---------------------------------------------------------------------------
template <class T>
struct PointDerivs {
    T u[3];
    T gl[3];
    T gu[3][3];
    T gs[3];
    T lap[3];
    T gd[3];
};

template <class T, int NF>
__device__ __forceinline__ void rhs_point(const PointDerivs<T> &d, const Coef<T> &c, T *out)
{
    const T div = d.gu[0][0] + d.gu[1][1] + d.gu[2][2];
    // Eq. 1
    out[0] = -(d.u[0] * d.gl[0] + d.u[1] * d.gl[1] + d.u[2] * d.gl[2]) - div;
    // Eq. 3 and Eq. 2:  2 (S . grad lnrho)_i
    //   = sum_j (d_j u_i + d_i u_j) d_j lnrho - (2/3) div d_i lnrho
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        T adv = d.u[0] * d.gu[i][0] + d.u[1] * d.gu[i][1] + d.u[2] * d.gu[i][2];
        T s2 = (d.gu[i][0] + d.gu[0][i]) * d.gl[0] + (d.gu[i][1] + d.gu[1][i]) * d.gl[1] +
               (d.gu[i][2] + d.gu[2][i]) * d.gl[2];
        T visc = c.nu * (d.lap[i] + s2) + c.nu3 * d.gd[i] - c.nu23 * div * d.gl[i];
        out[1 + i] = -adv - c.cs2 * d.gl[i] + visc;
    }
    if (NF == 5)
        out[4] = -(d.u[0] * d.gs[0] + d.u[1] * d.gs[1] + d.u[2] * d.gs[2]);
}

// Eq. 10 update of one value: w <- alpha w + dt r (the first substep ignores
// the old w, alpha_1 = 0), u_out <- u + beta w; arithmetic in TA.
template <class TA, class TW, class TS>
__device__ __forceinline__ void rk3_update(bool first, TA alpha, TA beta, TA dt, TA r, TS u,
                                           TW &w, TS &out)
{
    TA wn = first ? dt * r : alpha * (TA)w + dt * r;
    w = (TW)wn;
    out = (TS)((TA)u + beta * wn);
}

// A value carried as an unevaluated sum of two FP32 numbers, hi + lo with
// |lo| <= ulp(hi) / 2 ("float-float", Dekker 1971): the precision form's
// Eq. 10 update in compensated FP32 arithmetic.  Built from an FP64 value
// (the RK3 coefficients and dt) or from an FP32 one (lo = 0).
struct ffloat {
    float hi, lo;
    __host__ __device__ ffloat() : hi(0.f), lo(0.f) {}
    __host__ __device__ ffloat(double v) : hi((float)v), lo((float)(v - (double)(float)v)) {}
};

// Error-free transformations (round-to-nearest FP32; explicit _rn operations
// so that nothing is contracted into a fused multiply-add):
// a * b = p + e exactly (fused multiply-add form of Dekker's product) ...
__device__ __forceinline__ void two_prod(float a, float b, float &p, float &e)
{
    p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
}
// ... a + b = s + e exactly (Knuth's TwoSum, no ordering of a and b needed) ...
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// ... and a + b = s + e exactly when |a| >= |b| (Dekker's FastTwoSum).
__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}

// Eq. 10 for one FP32 value in float-float arithmetic: w_new = alpha w + dt r
// kept as hi + lo (the products and their sum error-free, the low-order
// terms summed in FP32), w stored as its FP32 rounding hi, and
// u_out = u + beta (hi + lo) rounded once to FP32 from an error-free sum.
// About 48 significant bits, so the result matches the FP64 update of the
// same inputs except where the two roundings of a near-tie differ.
__device__ __forceinline__ void rk3_update_ff(bool first, ffloat alpha, ffloat beta, ffloat dt,
                                              float r, float u, float &w, float &out)
{
    float p2, e2, hi, lo;
    two_prod(dt.hi, r, p2, e2);
    e2 = __fmaf_rn(dt.lo, r, e2);
    if (first) {
        fast_two_sum(p2, e2, hi, lo);
    } else {
        float p1, e1, s, t;
        two_prod(alpha.hi, w, p1, e1);
        e1 = __fmaf_rn(alpha.lo, w, e1);
        two_sum(p1, p2, s, t);
        // s can be small after cancellation: renormalise with the full TwoSum
        two_sum(s, __fadd_rn(t, __fadd_rn(e1, e2)), hi, lo);
    }
    w = hi;
    float q, f, s2, t2;
    two_prod(beta.hi, hi, q, f);
    f = __fmaf_rn(beta.hi, lo, f);
    f = __fmaf_rn(beta.lo, hi, f);
    two_sum(u, q, s2, t2);
    out = __fadd_rn(s2, __fadd_rn(t2, f));
}

template <>
__device__ __forceinline__ void rk3_update<ffloat, float, float>(bool first, ffloat alpha,
                                                                 ffloat beta, ffloat dt, ffloat r,
                                                                 float u, float &w, float &out)
{
    rk3_update_ff(first, alpha, beta, dt, r.hi, u, w, out);
}

// Exact IEEE-754 conversions between binary32 and binary64 done with integer
// instructions, so that GB300's narrow FP64 pipe is left to the arithmetic.
// binary32 (sign, 8-bit exponent e, 23-bit fraction m) -> binary64: exponent
// e + 896 (= e - 127 + 1023), fraction m << 29.  binary64 -> binary32: exponent
// E - 896, the top 23 fraction bits, rounded to nearest, ties to even, on the
// 29 dropped bits (a carry out of the fraction bumps the exponent, and past
// the largest finite value gives infinity, as round-to-nearest requires).
// Zero, subnormal, infinite and NaN operands, and results below the normal
// binary32 range, take the hardware conversion.
__device__ __forceinline__ double f32_to_f64_int(float x)
{
    const uint32_t b = __float_as_uint(x);
    const uint32_t e = (b >> 23) & 0xffu;
    if (e == 0u || e == 0xffu)
        return (double)x;
    const uint32_t hi = (b & 0x80000000u) | ((e + 896u) << 20) | ((b & 0x7fffffu) >> 3);
    return __hiloint2double((int)hi, (int)(b << 29));
}

__device__ __forceinline__ float f64_to_f32_int(double v)
{
    const uint32_t hi = (uint32_t)__double2hiint(v), lo = (uint32_t)__double2loint(v);
    const int e = (int)((hi >> 20) & 0x7ffu) - 896;
    if (e <= 0 || e >= 255)
        return __double2float_rn(v);
    const uint32_t m = ((hi & 0xfffffu) << 3) | (lo >> 29);
    const uint32_t rest = lo & 0x1fffffffu;
    const uint32_t up = (rest > 0x10000000u) || (rest == 0x10000000u && (m & 1u));
    return __uint_as_float(((hi & 0x80000000u) | ((uint32_t)e << 23) | m) + up);
}

// Eq. 10 in FP64 for FP32 state: the same arithmetic with explicit fused
// multiply-adds whichever conversions are used (ICVT: the integer routines
// above, else the hardware conversions), so the two give identical bits.
template <bool ICVT, class TW>
__device__ __forceinline__ void rk3_update_f64(bool first, double alpha, double beta, double dt,
                                               float r, float u, TW &w, float &out)
{
    auto up = [](float v) { return ICVT ? f32_to_f64_int(v) : (double)v; };
    auto down = [](double v) { return ICVT ? f64_to_f32_int(v) : __double2float_rn(v); };
    const double rd = up(r);
    double wd;
    if constexpr (sizeof(TW) == 8)
        wd = w;
    else
        wd = up(w);
    const double wn = first ? dt * rd : fma(alpha, wd, dt * rd);
    if constexpr (sizeof(TW) == 8)
        w = wn;
    else
        w = down(wn);
    out = down(fma(beta, wn, up(u)));
}

// Store v at interior (x, y, z) of field f and at its periodic ghost copies.
template <class T>
__device__ __forceinline__ void store_ghosted(T *base, const Layout &L, int f, int z, int y, int x,
                                              T v)
{
    const long long i0 = lidx(L, f, z, y, x);
    base[i0] = v;
    long long dx = 0, dy = 0;
    if (x < GX)
        dx = L.nx;
    else if (x >= L.nx - GX)
        dx = -L.nx;
    if (y < GY)
        dy = (long long)L.ny * L.P;
    else if (y >= L.ny - GY)
        dy = -(long long)L.ny * L.P;
    if (dx)
        base[i0 + dx] = v;
    if (dy) {
        base[i0 + dy] = v;
        if (dx)
            base[i0 + dy + dx] = v;
    }
}

// Host-side launch helpers implemented in the kernel translation units.
struct StateBufs {
    void *in;    // padded state, storage type
    void *out;   // padded state, storage type
    void *w;     // padded 2N register (u-tilde)
    void *div;   // padded divergence field (19-point form)
    Layout Ls;   // layout of in/out/div (div uses one field)
    Layout Lw;   // layout of w
};

}  // namespace gbfd
