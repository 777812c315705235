// Derivative gathering for one grid point (Eqs. 6-8), written against an
// accessor A(f, dz, dy, dx) that returns field f at the given offset from
// the point.  Used by the simple kernels (global-memory accessor) and by
// the tiled kernels (shared-memory accessor) so that both evaluate the same
// operators in the same order.
#pragma once

#include "common.cuh"

namespace gbfd {

template <class T, class Acc>
__device__ __forceinline__ T d1_axis(const Acc &A, int f, int axis, const Coef<T> &c)
{
    T acc = (T)0;
#pragma unroll
    for (int k = 1; k <= 3; ++k) {
        T p, m;
        if (axis == 0) {
            p = A(f, 0, 0, k);
            m = A(f, 0, 0, -k);
        } else if (axis == 1) {
            p = A(f, 0, k, 0);
            m = A(f, 0, -k, 0);
        } else {
            p = A(f, k, 0, 0);
            m = A(f, -k, 0, 0);
        }
        acc += c.d1[axis][k - 1] * (p - m);
    }
    return acc;
}

template <class T, class Acc>
__device__ __forceinline__ T d2_axis(const Acc &A, int f, int axis, T centre, const Coef<T> &c)
{
    T acc = c.d2c[axis] * centre;
#pragma unroll
    for (int k = 1; k <= 3; ++k) {
        T p, m;
        if (axis == 0) {
            p = A(f, 0, 0, k);
            m = A(f, 0, 0, -k);
        } else if (axis == 1) {
            p = A(f, 0, k, 0);
            m = A(f, 0, -k, 0);
        } else {
            p = A(f, k, 0, 0);
            m = A(f, -k, 0, 0);
        }
        acc += c.d2[axis][k - 1] * (p + m);
    }
    return acc;
}

// Bidiagonal mixed derivative (Eq. 8) in pair p: 0 = (x,y), 1 = (x,z), 2 = (y,z).
template <class T, class Acc>
__device__ __forceinline__ T dmix_pair(const Acc &A, int f, int p, const Coef<T> &c)
{
    T acc = (T)0;
#pragma unroll
    for (int k = 1; k <= 3; ++k) {
        T pp, mp, mm, pm;  // (+a,+b), (-a,+b), (-a,-b), (+a,-b)
        if (p == 0) {
            pp = A(f, 0, k, k);
            mp = A(f, 0, k, -k);
            mm = A(f, 0, -k, -k);
            pm = A(f, 0, -k, k);
        } else if (p == 1) {
            pp = A(f, k, 0, k);
            mp = A(f, k, 0, -k);
            mm = A(f, -k, 0, -k);
            pm = A(f, -k, 0, k);
        } else {
            pp = A(f, k, k, 0);
            mp = A(f, k, -k, 0);
            mm = A(f, -k, -k, 0);
            pm = A(f, -k, k, 0);
        }
        acc += c.mx[p][k - 1] * ((pp - mp) + (mm - pm));
    }
    return acc;
}

// All derivatives the right-hand side needs at one point.  MIXED = true is
// the 55-point form (grad div u from Eq. 7 + Eq. 8); MIXED = false leaves
// gd = 0 (first pass of the 19-point form).
template <class T, int NF, bool MIXED, class Acc>
__device__ __forceinline__ void gather_derivs(const Acc &A, const Coef<T> &c, PointDerivs<T> &d)
{
#pragma unroll
    for (int i = 0; i < 3; ++i)
        d.u[i] = A(1 + i, 0, 0, 0);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        d.gl[a] = d1_axis(A, 0, a, c);
#pragma unroll
        for (int i = 0; i < 3; ++i)
            d.gu[i][a] = d1_axis(A, 1 + i, a, c);
        d.gs[a] = (NF == 5) ? d1_axis(A, 4, a, c) : (T)0;
    }
    T d2u[3][3];  // d2u[i][a] = D2 along axis a of u_i
#pragma unroll
    for (int i = 0; i < 3; ++i) {
#pragma unroll
        for (int a = 0; a < 3; ++a)
            d2u[i][a] = d2_axis(A, 1 + i, a, d.u[i], c);
        d.lap[i] = d2u[i][0] + d2u[i][1] + d2u[i][2];
    }
    if (MIXED) {
        // d_i(div u) = sum_j d_i d_j u_j
        d.gd[0] = d2u[0][0] + dmix_pair(A, 2, 0, c) + dmix_pair(A, 3, 1, c);
        d.gd[1] = dmix_pair(A, 1, 0, c) + d2u[1][1] + dmix_pair(A, 3, 2, c);
        d.gd[2] = dmix_pair(A, 1, 1, c) + dmix_pair(A, 2, 2, c) + d2u[2][2];
    } else {
        d.gd[0] = d.gd[1] = d.gd[2] = (T)0;
    }
}

}  // namespace gbfd
