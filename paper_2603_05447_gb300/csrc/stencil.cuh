// stencil.cuh -- device building blocks shared by the stencil kernels of
// libgpeshell (steps, batches, adjoint): the packed segment layout, the
// per-warp brick tile and its 7-point Laplacian (Eq. (B1)), the ramp
// schedule and small reductions.  Not part of the ABI.
#pragma once

#include "gpe_internal.cuh"

#include <type_traits>

namespace gpe {

// Stencil kernels run one brick per warp; a block holds NW warps, each with
// its own shared-memory workspace (brick tile with face halo, the 7 brick
// records and the list of stored segments), passed as dynamic shared memory.
#ifndef GPE_NW_F
#define GPE_NW_F 8
#endif
// fetch the records of a warp's next brick while it processes the current one
#ifndef GPE_REC_AHEAD
#define GPE_REC_AHEAD 1
#endif
template <typename R>
struct KernelCfg {
    static constexpr int NW = sizeof(R) == 4 ? GPE_NW_F : 4;  // warps per block
    static constexpr int THREADS = 32 * NW;
};

// Minimum resident blocks per SM requested from the register allocator:
// as many as the shared-memory workspaces allow (228 KiB per SM, 1 KiB
// reserved per block), at most GPE_MINB_F (single precision) / GPE_MINB_D
// (double precision, whose kernels need more registers).
#ifndef GPE_MINB_F
#define GPE_MINB_F 4
#endif
#ifndef GPE_MINB_D
#define GPE_MINB_D 3
#endif
#define GPE_BOUNDS(R) __launch_bounds__(KernelCfg<R>::THREADS, (min_blocks<R, BX, BY, BZ>()))
// kernels templated on the stencil NP: the 19-point form needs more
// registers; in single precision three blocks an SM (80 registers) beat two
// (about 105) despite a few spilled bytes in some variants
#define GPE_BOUNDS_NP(R) \
    __launch_bounds__(KernelCfg<R>::THREADS, (NP == 19 ? (sizeof(R) == 4 ? 3 : 2) : min_blocks<R, BX, BY, BZ>()))

// ------------------------------------------------------------ packed layout
// supported brick shapes (shape id, BX, BY, BZ)
#define GPE_SHAPES(M) \
    M(0, 8, 8, 8)     \
    M(1, 8, 8, 4)     \
    M(2, 8, 4, 4)

struct GridView {
    const int32_t *nbr;
    const BrickRec *rec;
    const BrickRec *rec7;   // per brick: its record, then its six face neighbours' (empty if absent)
    int64_t nb;
    const BrickRec *rec19;  // 19-point grids: the record, 6 face and 12 edge neighbours' records
};

inline GridView view(const gpe_grid *g) { return GridView{g->d_nbr, g->d_rec, g->d_rec7, g->nb, g->d_rec19}; }

// segment geometry of a brick shape (BX must be 8: two segments per row)
template <int BX, int BY, int BZ>
struct Seg {
    static_assert(BX == 8, "bricks are 8 cells long in x");
    static constexpr int SX = BX / 4;          // segments per x-row
    static constexpr int PLANE = SX * BY;      // segments per z-plane (divides 32)
    static constexpr int NSEG = PLANE * BZ;    // segments per brick
    static constexpr int NIT = NSEG / 32;      // warp iterations per brick
    static_assert(32 % PLANE == 0 && NSEG % 32 == 0, "brick shape must tile the warp");
};

// Values are complex (float2, double2) or, for real-valued imaginary-time
// states, real (float, double); these helpers serve both.
template <typename CT>
__host__ __device__ constexpr bool is_cplx()
{
    return !std::is_arithmetic<CT>::value;
}
template <typename CT>
struct RealOf {
    using T = CT;
};
template <>
struct RealOf<float2> {
    using T = float;
};
template <>
struct RealOf<double2> {
    using T = double;
};

// Packed single-precision pairs: the f32x2 add / multiply / fused
// multiply-add instructions of sm_100 and later act on both halves of a
// 64-bit register pair, i.e. on the real and imaginary parts of a complex64
// value at once, each half rounded exactly as the scalar instruction would
// round it.  They halve the arithmetic instruction count of the complex64
// stencils without changing any result.
__device__ __forceinline__ unsigned long long f2pk(float2 a)
{
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a.x), "f"(a.y));
    return r;
}
__device__ __forceinline__ float2 f2up(unsigned long long r)
{
    float2 a;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a.x), "=f"(a.y) : "l"(r));
    return a;
}
__device__ __forceinline__ float2 add2(float2 a, float2 b)
{
    unsigned long long d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2pk(a)), "l"(f2pk(b)));
    return f2up(d);
}
__device__ __forceinline__ float2 sub2(float2 a, float2 b)  // a - b
{
    unsigned long long d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2pk(a)), "l"(f2pk(b)));
    return f2up(d);
}
__device__ __forceinline__ float2 mul2(float2 a, float2 b)
{
    unsigned long long d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2pk(a)), "l"(f2pk(b)));
    return f2up(d);
}
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c)  // a * b + c, one rounding per half
{
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(f2pk(a)), "l"(f2pk(b)), "l"(f2pk(c)));
    return f2up(d);
}
__device__ __forceinline__ float2 dup2(float f) { return make_float2(f, f); }

template <typename CT>
__device__ __forceinline__ CT czero()
{
    if constexpr (is_cplx<CT>()) {
        CT z;
        z.x = 0;
        z.y = 0;
        return z;
    } else {
        return CT(0);
    }
}
// |v|^2
template <typename CT>
__device__ __forceinline__ typename RealOf<CT>::T norm2(const CT &v)
{
    if constexpr (is_cplx<CT>())
        return v.x * v.x + v.y * v.y;
    else
        return v * v;
}
// v * f, f real
__device__ __forceinline__ float2 scale(float2 v, float f) { return mul2(v, dup2(f)); }
template <typename CT, typename R>
__device__ __forceinline__ CT scale(CT v, R f)
{
    if constexpr (is_cplx<CT>()) {
        v.x *= f;
        v.y *= f;
        return v;
    } else {
        return v * f;
    }
}
// c + a L, a real
__device__ __forceinline__ float2 axpy(const float2 &c, float a, const float2 &L) { return fma2(dup2(a), L, c); }
__device__ __forceinline__ float axpy(float c, float a, float L) { return __fmaf_rn(a, L, c); }
template <typename CT, typename R>
__device__ __forceinline__ CT axpy(const CT &c, R a, const CT &L)
{
    if constexpr (is_cplx<CT>()) {
        CT o;
        o.x = c.x + a * L.x;
        o.y = c.y + a * L.y;
        return o;
    } else {
        return c + a * L;
    }
}
// Re(conj(a) b)
template <typename CT>
__device__ __forceinline__ typename RealOf<CT>::T dotre(const CT &a, const CT &b)
{
    if constexpr (is_cplx<CT>())
        return a.x * b.x + a.y * b.y;
    else
        return a * b;
}
template <typename CT>
__device__ __forceinline__ bool finite_v(const CT &v)
{
    if constexpr (is_cplx<CT>())
        return isfinite(v.x) && isfinite(v.y);
    else
        return isfinite(v);
}
__device__ __forceinline__ float2 vadd(const float2 &a, const float2 &b) { return add2(a, b); }
template <typename CT>
__device__ __forceinline__ CT vadd(const CT &a, const CT &b)
{
    if constexpr (is_cplx<CT>()) {
        CT o;
        o.x = a.x + b.x;
        o.y = a.y + b.y;
        return o;
    } else {
        return a + b;
    }
}
// L + wxy exy + wxz exz + wyz eyz: the edge terms of App. B's 19-point
// stencil added to its face-and-centre part
__device__ __forceinline__ float2 edgev(const float2 &L, const float2 &exy, const float2 &exz, const float2 &eyz,
                                        float wxy, float wxz, float wyz)
{
    return fma2(dup2(wyz), eyz, fma2(dup2(wxz), exz, fma2(dup2(wxy), exy, L)));
}
__device__ __forceinline__ float edgev(float L, float exy, float exz, float eyz, float wxy, float wxz, float wyz)
{
    return __fmaf_rn(wyz, eyz, __fmaf_rn(wxz, exz, __fmaf_rn(wxy, exy, L)));
}
template <typename CT, typename R>
__device__ __forceinline__ CT edgev(const CT &L, const CT &exy, const CT &exz, const CT &eyz, R wxy, R wxz, R wyz)
{
    if constexpr (is_cplx<CT>()) {
        CT o;
        o.x = L.x + wxy * exy.x + wxz * exz.x + wyz * eyz.x;
        o.y = L.y + wxy * exy.y + wxz * exz.y + wyz * eyz.y;
        return o;
    } else {
        return L + wxy * exy + wxz * exz + wyz * eyz;
    }
}
// one component of the 7-point Laplacian (Eq. (B1)) from opposite-neighbour
// sums: (x- + x+)/hx^2 + (y- + y+)/hy^2 + (z- + z+)/hz^2 - c6 c.  In single
// precision the order of the roundings is fixed explicitly, the same as the
// packed complex64 form (lapv below), so that a real-valued float state and a
// complex64 state with zero imaginary part compute bit-identical values.
__device__ __forceinline__ float lap1(float xp, float xm, float yp, float ym, float zp, float zm, float c, float ihx2,
                                      float ihy2, float ihz2, float c6)
{
    float t = __fmul_rn(__fadd_rn(xp, xm), ihx2);
    t = __fmaf_rn(__fadd_rn(yp, ym), ihy2, t);
    t = __fmaf_rn(__fadd_rn(zp, zm), ihz2, t);
    return __fmaf_rn(-c6, c, t);
}
template <typename R>
__device__ __forceinline__ R lap1(R xp, R xm, R yp, R ym, R zp, R zm, R c, R ihx2, R ihy2, R ihz2, R c6)
{
    return (xp + xm) * ihx2 + (yp + ym) * ihy2 + (zp + zm) * ihz2 - c6 * c;
}
// complex64: the same operations as lap1 on both parts at once
__device__ __forceinline__ float2 lapv(const float2 &xp, const float2 &xm, const float2 &yp, const float2 &ym,
                                       const float2 &zp, const float2 &zm, const float2 &c, float ihx2, float ihy2,
                                       float ihz2, float c6)
{
    float2 t = mul2(add2(xp, xm), dup2(ihx2));
    t = fma2(add2(yp, ym), dup2(ihy2), t);
    t = fma2(add2(zp, zm), dup2(ihz2), t);
    return fma2(dup2(-c6), c, t);
}
template <typename CT, typename R>
__device__ __forceinline__ CT lapv(const CT &xp, const CT &xm, const CT &yp, const CT &ym, const CT &zp, const CT &zm,
                                   const CT &c, R ihx2, R ihy2, R ihz2, R c6)
{
    if constexpr (is_cplx<CT>()) {
        CT L;
        L.x = lap1(xp.x, xm.x, yp.x, ym.x, zp.x, zm.x, c.x, ihx2, ihy2, ihz2, c6);
        L.y = lap1(xp.y, xm.y, yp.y, ym.y, zp.y, zm.y, c.y, ihx2, ihy2, ihz2, c6);
        return L;
    } else {
        return lap1(xp, xm, yp, ym, zp, zm, c, ihx2, ihy2, ihz2, c6);
    }
}

__device__ __forceinline__ float2 shfl_up(float2 v, int d)
{
    v.x = __shfl_up_sync(0xffffffffu, v.x, d);
    v.y = __shfl_up_sync(0xffffffffu, v.y, d);
    return v;
}
__device__ __forceinline__ double2 shfl_up(double2 v, int d)
{
    v.x = __shfl_up_sync(0xffffffffu, v.x, d);
    v.y = __shfl_up_sync(0xffffffffu, v.y, d);
    return v;
}
__device__ __forceinline__ float2 shfl_down(float2 v, int d)
{
    v.x = __shfl_down_sync(0xffffffffu, v.x, d);
    v.y = __shfl_down_sync(0xffffffffu, v.y, d);
    return v;
}
__device__ __forceinline__ double2 shfl_down(double2 v, int d)
{
    v.x = __shfl_down_sync(0xffffffffu, v.x, d);
    v.y = __shfl_down_sync(0xffffffffu, v.y, d);
    return v;
}
__device__ __forceinline__ float2 shfl_xor(float2 v, int d)
{
    v.x = __shfl_xor_sync(0xffffffffu, v.x, d);
    v.y = __shfl_xor_sync(0xffffffffu, v.y, d);
    return v;
}
__device__ __forceinline__ double2 shfl_xor(double2 v, int d)
{
    v.x = __shfl_xor_sync(0xffffffffu, v.x, d);
    v.y = __shfl_xor_sync(0xffffffffu, v.y, d);
    return v;
}

// 4 consecutive complex values (one segment, 32-byte aligned) with 256-bit
// accesses, so that each lane moves whole 32-byte sectors; CG: read through
// L2 only (data written by other blocks of the same launch)
template <bool CG>
__device__ __forceinline__ void ld4(const float2 *p, float2 (&v)[4])
{
    float a[8];
    if (CG)
        asm volatile("ld.global.cg.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                     : "=f"(a[0]), "=f"(a[1]), "=f"(a[2]), "=f"(a[3]), "=f"(a[4]), "=f"(a[5]), "=f"(a[6]), "=f"(a[7])
                     : "l"(p));
    else
        asm volatile("ld.global.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                     : "=f"(a[0]), "=f"(a[1]), "=f"(a[2]), "=f"(a[3]), "=f"(a[4]), "=f"(a[5]), "=f"(a[6]), "=f"(a[7])
                     : "l"(p));
#pragma unroll
    for (int i = 0; i < 4; ++i) v[i] = make_float2(a[2 * i], a[2 * i + 1]);
}
template <bool CG>
__device__ __forceinline__ void ld4(const double2 *p, double2 (&v)[4])
{
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        double a0, a1, a2, a3;
        if (CG)
            asm volatile("ld.global.cg.v4.f64 {%0,%1,%2,%3}, [%4];"
                         : "=d"(a0), "=d"(a1), "=d"(a2), "=d"(a3) : "l"(p + 2 * h));
        else
            asm volatile("ld.global.v4.f64 {%0,%1,%2,%3}, [%4];" : "=d"(a0), "=d"(a1), "=d"(a2), "=d"(a3) : "l"(p + 2 * h));
        v[2 * h] = make_double2(a0, a1);
        v[2 * h + 1] = make_double2(a2, a3);
    }
}
__device__ __forceinline__ void st4(float2 *p, const float2 (&v)[4])
{
    asm volatile("st.global.v8.f32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"l"(p), "f"(v[0].x), "f"(v[0].y), "f"(v[1].x),
                 "f"(v[1].y), "f"(v[2].x), "f"(v[2].y), "f"(v[3].x), "f"(v[3].y)
                 : "memory");
}
__device__ __forceinline__ void st4(double2 *p, const double2 (&v)[4])
{
#pragma unroll
    for (int h = 0; h < 2; ++h)
        asm volatile("st.global.v4.f64 [%0], {%1,%2,%3,%4};" ::"l"(p + 2 * h), "d"(v[2 * h].x), "d"(v[2 * h].y),
                     "d"(v[2 * h + 1].x), "d"(v[2 * h + 1].y)
                     : "memory");
}
// 4 consecutive reals of a real-valued state (one segment, 16- or 32-byte
// aligned); CG as for ld4 above
template <bool CG>
__device__ __forceinline__ void ld4(const float *p, float (&v)[4])
{
    if (CG)
        asm volatile("ld.global.cg.v4.f32 {%0,%1,%2,%3}, [%4];" : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]) : "l"(p));
    else
        asm volatile("ld.global.v4.f32 {%0,%1,%2,%3}, [%4];" : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]) : "l"(p));
}
template <bool CG>
__device__ __forceinline__ void ld4(const double *p, double (&v)[4])
{
    if (CG)
        asm volatile("ld.global.cg.v4.f64 {%0,%1,%2,%3}, [%4];" : "=d"(v[0]), "=d"(v[1]), "=d"(v[2]), "=d"(v[3]) : "l"(p));
    else
        asm volatile("ld.global.v4.f64 {%0,%1,%2,%3}, [%4];" : "=d"(v[0]), "=d"(v[1]), "=d"(v[2]), "=d"(v[3]) : "l"(p));
}
__device__ __forceinline__ void st4(float *p, const float (&v)[4])
{
    asm volatile("st.global.v4.f32 [%0], {%1,%2,%3,%4};" ::"l"(p), "f"(v[0]), "f"(v[1]), "f"(v[2]), "f"(v[3]) : "memory");
}
__device__ __forceinline__ void st4(double *p, const double (&v)[4])
{
    asm volatile("st.global.v4.f64 [%0], {%1,%2,%3,%4};" ::"l"(p), "d"(v[0]), "d"(v[1]), "d"(v[2]), "d"(v[3]) : "memory");
}

// 4 consecutive reals (16- or 32-byte aligned), read-only data
__device__ __forceinline__ void ldr4(const float *p, float (&v)[4])
{
    const float4 a = __ldg(reinterpret_cast<const float4 *>(p));
    v[0] = a.x;
    v[1] = a.y;
    v[2] = a.z;
    v[3] = a.w;
}
__device__ __forceinline__ void ldr4(const double *p, double (&v)[4])
{
    asm volatile("ld.global.nc.v4.f64 {%0,%1,%2,%3}, [%4];" : "=d"(v[0]), "=d"(v[1]), "=d"(v[2]), "=d"(v[3]) : "l"(p));
}

struct Identity {
    template <typename CT>
    __device__ __forceinline__ CT operator()(CT v, uint32_t) const { return v; }
};

template <bool CG, typename CT>
__device__ __forceinline__ CT ld1(const CT *p)
{
    return CG ? __ldcg(p) : *p;
}

// Per-warp workspace.  The brick's segments, with the y and z face halos as
// whole rows (rows y = -1..BY, planes z = -1..BZ), are stored as UPS planes of
// 16-byte units: unit u of every segment slot is contiguous, so lanes that
// take consecutive segments touch consecutive 16-byte units (no shared-memory
// bank conflicts).  The x face halos are separate columns.  Then the records
// of the brick and its six face neighbours and the brick's stored segments in
// order, each as its tile slot and x-halo row (slot | h << 8).  The records of the warp's next brick are fetched into nrec while
// the current brick is processed.
template <typename CT, int BX, int BY, int BZ, int NP = 7>
struct WarpSpace {
    static constexpr int SX = BX / 4, TY = BY + 2, TZ = BZ + 2;
    // records: own and 6 face neighbours (7-point), and 12 edge neighbours
    // (19-point); x-halo columns: rows y in [0, BY) x z in [0, BZ), or with
    // the halo rows y = -1, BY and planes z = -1, BZ for the 19-point stencil
    static constexpr int NR = NP == 19 ? 19 : 7;
    static constexpr int XH = NP == 19 ? TY * TZ : BY * BZ;
    static constexpr int NSLOT = SX * TY * TZ;                   // segment slots incl. y/z halos
    static constexpr int UPS = (int)(4 * sizeof(CT) / 16);       // 16-byte units per segment
    // plane stride (in units) = 4 (UPS 2) or 2 (UPS 4) mod 8: the UPS units of
    // one segment fall in distinct 16-byte bank groups, so UPS lanes can fill
    // one segment's units in one conflict-free access
    static constexpr int PSTR = NSLOT + (((UPS == 2 ? 4 : 2) - NSLOT % 8) + 8) % 8;
    static constexpr int CPU_ = 4 / UPS;                         // cells per unit
    static constexpr int NSEG = Seg<BX, BY, BZ>::NSEG;
    static constexpr int ROW = SX, PLANE = SX * TY;              // slot strides in y and z
    __device__ __forceinline__ static int slot(int hx, int y, int z) { return hx + SX * ((y + 1) + TY * (z + 1)); }
    __device__ __forceinline__ static int h(int y, int z) { return NP == 19 ? (y + 1) + TY * (z + 1) : y + BY * z; }
    uint4 units[UPS][PSTR];
    // x halos: per row (for the 19-point stencil also on the halo rows and
    // planes) the 16-byte unit of the neighbour segment that holds the halo
    // cell (cell 3 of the -x brick's last segment of the row, cell 0 of the
    // +x brick's first), filled by cp.async like the tile.
    static constexpr int XW = 16;
    alignas(16) unsigned char xlo_[XH * XW];  // x = -1
    alignas(16) unsigned char xhi_[XH * XW];  // x = BX
    __device__ __forceinline__ CT xm_cell(int h) const  // the cell at x = -1 of row h
    {
        return reinterpret_cast<const CT *>(xlo_ + h * XW)[CPU_ - 1];
    }
    __device__ __forceinline__ CT xp_cell(int h) const  // the cell at x = BX of row h
    {
        return reinterpret_cast<const CT *>(xhi_ + h * XW)[0];
    }
    __device__ __forceinline__ CT *xm_slot(int h) { return reinterpret_cast<CT *>(xlo_ + h * XW) + (CPU_ - 1); }
    __device__ __forceinline__ CT *xp_slot(int h) { return reinterpret_cast<CT *>(xhi_ + h * XW); }
    alignas(16) BrickRec rec[NR];
#if GPE_REC_AHEAD
    BrickRec nrec[NR];  // records of the warp's next brick, fetched ahead
    long long nrec_b;  // brick whose records nrec holds (-1: none)
    uint16_t list[NSEG];
    uint8_t pad[(16 - ((2 * NSEG + 8) % 16)) % 16];
#else
    uint16_t list[NSEG];
    uint8_t pad[(16 - ((2 * NSEG) % 16)) % 16];
#endif

    __device__ __forceinline__ void get(int s, CT (&v)[4]) const
    {
#pragma unroll
        for (int u = 0; u < UPS; ++u) {
            const uint4 w = units[u][s];
            const CT *c = reinterpret_cast<const CT *>(&w);
#pragma unroll
            for (int i = 0; i < CPU_; ++i) v[u * CPU_ + i] = c[i];
        }
    }
    __device__ __forceinline__ void put(int s, const CT (&v)[4])
    {
#pragma unroll
        for (int u = 0; u < UPS; ++u) {
            uint4 w;
            CT *c = reinterpret_cast<CT *>(&w);
#pragma unroll
            for (int i = 0; i < CPU_; ++i) c[i] = v[u * CPU_ + i];
            units[u][s] = w;
        }
    }
    __device__ __forceinline__ CT first(int s) const  // cell 0 of slot s
    {
        return reinterpret_cast<const CT *>(&units[0][s])[0];
    }
    __device__ __forceinline__ CT last(int s) const  // cell 3 of slot s
    {
        return reinterpret_cast<const CT *>(&units[UPS - 1][s])[CPU_ - 1];
    }
};

template <typename R, int BX, int BY, int BZ, typename CT = typename Cx<R>::T, int NP = 7>
constexpr size_t smem_bytes()
{
    return (size_t)KernelCfg<R>::NW * sizeof(WarpSpace<CT, BX, BY, BZ, NP>);
}

// the calling warp's workspace (call once per kernel: it resets the
// next-record tag)
template <typename R, int BX, int BY, int BZ>
constexpr int min_blocks()
{
    const int cap = sizeof(R) == 4 ? GPE_MINB_F : GPE_MINB_D;
    const int fit = (int)((228u * 1024u) / (smem_bytes<R, BX, BY, BZ>() + 1024u));
    return fit < 1 ? 1 : (fit < cap ? fit : cap);
}

template <typename R, int BX, int BY, int BZ, typename CT = typename Cx<R>::T, int NP = 7>
__device__ __forceinline__ WarpSpace<CT, BX, BY, BZ, NP> &warp_space()
{
    extern __shared__ __align__(16) unsigned char gpe_smem[];
    auto &ws = reinterpret_cast<WarpSpace<CT, BX, BY, BZ, NP> *>(gpe_smem)[threadIdx.x >> 5];
#if GPE_REC_AHEAD
    if ((threadIdx.x & 31) == 0) ws.nrec_b = -1;
    __syncwarp();
#endif
    return ws;
}

template <typename CT>
__device__ __forceinline__ void put4(CT *t, const CT (&v)[4])
{
    t[0] = v[0];
    t[1] = v[1];
    t[2] = v[2];
    t[3] = v[3];
}

// 16-byte asynchronous global -> shared copies (cp.async, L2 only): the tile
// fill issues every copy of a brick before waiting on any of them, so a warp
// keeps its whole tile (and its body's prefetched operands) in flight without
// staging them in registers.  valid == false writes 16 zero bytes.
__device__ __forceinline__ void cp_async16(void *dst, const void *src, bool valid)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(valid ? 16 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Records of brick b (slot 0), of its six face neighbours (slots 1..6,
// order -x +x -y +y -z +z) and, for the 19-point stencil, of its 12 edge
// neighbours (slots 7..18: xy, xz, yz edges; order as in the grid builder);
// an absent neighbour has an empty record.  One row (224 or 608 bytes) moved
// into ws.rec: from ws.nrec when it was fetched ahead, else from global
// memory.  Then the row of brick `next` (if >= 0) is fetched ahead into
// ws.nrec by cp.async; it completes with the tile's copies.
template <typename WS>
__device__ __forceinline__ void fetch_recs(WS &ws, const GridView &G, int64_t b, int64_t next)
{
    constexpr int NU = 2 * WS::NR;  // 16-byte words of one row of records
    const uint4 *rows = reinterpret_cast<const uint4 *>(WS::NR == 19 ? G.rec19 : G.rec7);
    const int lane = threadIdx.x & 31;
    cp_async_wait_all();
    __syncwarp();
#if GPE_REC_AHEAD
    const bool ahead = ws.nrec_b == (long long)b;
    for (int u = lane; u < NU; u += 32)
        reinterpret_cast<uint4 *>(ws.rec)[u] = ahead ? reinterpret_cast<const uint4 *>(ws.nrec)[u] : __ldg(rows + NU * b + u);
    __syncwarp();
    if (next >= 0)
        for (int u = lane; u < NU; u += 32) cp_async16(reinterpret_cast<uint4 *>(ws.nrec) + u, rows + NU * next + u, true);
    if (lane == 0) ws.nrec_b = next;
    __syncwarp();
#else
    (void)next;
    for (int u = lane; u < NU; u += 32) reinterpret_cast<uint4 *>(ws.rec)[u] = __ldg(rows + NU * b + u);
    __syncwarp();
#endif
}

// does the load transform XF provide a whole-segment form xf.seg(v, idx)?
template <typename XF, typename CT, typename = void>
struct HasSeg : std::false_type {};
template <typename XF, typename CT>
struct HasSeg<XF, CT, std::void_t<decltype(std::declval<const XF &>().seg(std::declval<CT (&)[4]>(), 0u))>>
    : std::true_type {};

// no operands to prefetch
struct NoPre {
    struct P {};
    __device__ __forceinline__ P operator()(uint32_t) const { return P{}; }
};

// Apply body(idx, pre, c, L) to every stored segment of brick b, one warp
// (next: the brick the warp takes after b, or -1):
// idx is the packed index of the segment's first cell, pre what load(idx)
// returned for it, c[4] its values and L[4] their 7-point Laplacians
// (Eq. (B1)), all taken from src after xf(value, packed index).  The warp
// stages the brick's stored segments (contiguous along the packed run) and
// the face halos from the neighbour bricks in its tile; absent cells read as
// zero.  Lanes then take the stored segments in order, so the packed indices
// of a warp's segments are consecutive and the bodies' own-cell loads and
// stores coalesce.  The first 32 segments' operands are loaded while the tile
// is in flight, the next 32's while a group is computed.  With xf the identity the tile is filled by cp.async;
// otherwise through registers, where xf is applied.
template <int BX, int BY, int BZ, bool CG, typename CT, int NP, typename R, typename XF, typename LOAD, typename BODY>
__device__ __forceinline__ void brick_apply(WarpSpace<CT, BX, BY, BZ, NP> &ws, const GridView &G, int64_t b,
                                            int64_t next, const CT *src, XF xf, R ihx2, R ihy2, R ihz2, LOAD load,
                                            BODY body)
{
    using S = Seg<BX, BY, BZ>;
    using W = WarpSpace<CT, BX, BY, BZ, NP>;
    constexpr bool ASYNC = std::is_same<XF, Identity>::value;
    const int lane = threadIdx.x & 31;
    fetch_recs(ws, G, b, next);
    const BrickRec &R0 = ws.rec[0];
    const int nst = __popc(R0.m[0]) + __popc(R0.m[1]) + __popc(R0.m[2]) + __popc(R0.m[3]);
    // unit u of one segment (4 cells; all units when u < 0) into tile slot sl
    auto seg_to = [&](const BrickRec &r, int q, int sl, int u) {
        uint32_t j = 0;
        const bool ok = seg_index(r, q, j);
        if constexpr (ASYNC) {
            const char *g = reinterpret_cast<const char *>(src + (ok ? j : 0u));
            cp_async16(&ws.units[u][sl], g + 16 * u, ok);
        } else {
            CT v[4];
            if (ok) {
                ld4<CG>(src + j, v);
                if constexpr (HasSeg<XF, CT>::value) {
                    xf.seg(v, j);
                } else {
#pragma unroll
                    for (int i = 0; i < 4; ++i) v[i] = xf(v[i], j + i);
                }
            } else {
#pragma unroll
                for (int i = 0; i < 4; ++i) v[i] = czero<CT>();
            }
            ws.put(sl, v);
        }
    };
    // ASYNC: UPS lanes per segment; else one lane per segment (u ignored)
    constexpr int LPS = ASYNC ? W::UPS : 1;
    // the stored segments in order (tile slot, x-halo row); with ASYNC the
    // unstored interior slots are zeroed here
    int nl = 0;
#pragma unroll
    for (int it = 0; it < S::NIT; ++it) {
        const int q = it * 32 + lane;
        const int y = (q / S::SX) % BY, z = q / S::PLANE;
        const int sl = W::slot(q % S::SX, y, z);
        const bool stored = (R0.m[q >> 5] >> (q & 31)) & 1u;
        const unsigned bal = __ballot_sync(0xffffffffu, stored);
        if (stored) {
            ws.list[nl + __popc(bal & ((1u << lane) - 1u))] = (uint16_t)(sl | (W::h(y, z) << 8));
        } else if constexpr (ASYNC) {
#pragma unroll
            for (int u = 0; u < W::UPS; ++u) ws.units[u][sl] = make_uint4(0, 0, 0, 0);
        }
        nl += __popc(bal);
    }
    // interior
    if constexpr (ASYNC) {
        // stored segments along the packed run: UPS lanes per segment, each
        // one contiguous 16-byte unit
        __syncwarp();
        const char *run = reinterpret_cast<const char *>(src + R0.off);
        for (int t = lane; t < nl * W::UPS; t += 32)
            cp_async16(&ws.units[t % W::UPS][ws.list[t / W::UPS] & 0xff], run + 16 * t, true);
    } else {
#pragma unroll
        for (int q = lane; q < S::NSEG; q += 32) seg_to(R0, q, W::slot(q % S::SX, (q / S::SX) % BY, q / S::PLANE), 0);
    }
    // -z / +z faces: whole segments of the neighbours' boundary planes
#pragma unroll
    for (int t = lane; t < 2 * S::PLANE * LPS; t += 32) {
        const int u = t / LPS, face = u / S::PLANE, qc = u % S::PLANE;
        seg_to(ws.rec[5 + face], face == 0 ? qc + S::PLANE * (BZ - 1) : qc,
               W::slot(qc % S::SX, qc / S::SX, face == 0 ? -1 : BZ), t % LPS);
    }
    // -y / +y faces: segments of the neighbours' boundary rows
#pragma unroll
    for (int t = lane; t < 2 * S::SX * BZ * LPS; t += 32) {
        const int u = t / LPS, face = u / (S::SX * BZ), v_ = u % (S::SX * BZ);
        const int hx = v_ % S::SX, z = v_ / S::SX;
        seg_to(ws.rec[3 + face], hx + S::SX * (face == 0 ? BY - 1 : 0) + S::PLANE * z,
               W::slot(hx, face == 0 ? -1 : BY, z), t % LPS);
    }
    // operands of the first 32 stored segments, while the tile is in flight
    typename std::decay<decltype(load(0u))>::type p0{};
    if (lane < nst) p0 = load(R0.off + 4u * (uint32_t)lane);
    if constexpr (NP == 19) {
        // y/z edge rows (y = -1 or BY, z = -1 or BZ) from the four yz-edge
        // neighbours (records 15..18: (0,-1,-1) (0,+1,-1) (0,-1,+1) (0,+1,+1))
#pragma unroll
        for (int t = lane; t < 4 * S::SX * LPS; t += 32) {
            const int v = t / LPS, e = v / S::SX, hx = v % S::SX;
            const int ys = (e & 1) ? 0 : BY - 1, zs = (e & 2) ? 0 : BZ - 1;
            seg_to(ws.rec[15 + e], hx + S::SX * ys + S::PLANE * zs,
                   W::slot(hx, (e & 1) ? BY : -1, (e & 2) ? BZ : -1), t % LPS);
        }
    }
    // -x / +x faces, identity transform: per row one 16-byte unit (the one
    // holding cell 3 of the -x brick's segment, or cell 0 of the +x brick's)
    // by cp.async; absent segments give a zero unit.  For the 19-point
    // stencil also the halo rows and planes, from the xy-edge (records
    // 7..10) and xz-edge (11..14) neighbours; the y-z corner rows, read by
    // no stencil, are zero.
    if constexpr (NP != 19 && ASYNC) {
        for (int u = lane; u < 2 * BY * BZ; u += 32) {
            const int face = u / (BY * BZ), v_ = u % (BY * BZ);
            const int y = v_ % BY, z = v_ / BY;
            uint32_t j = 0;
            const bool ok = seg_index(ws.rec[1 + face], (face == 0 ? S::SX - 1 : 0) + S::SX * y + S::PLANE * z, j);
            const char *g = reinterpret_cast<const char *>(src + (ok ? j : 0u)) + (face == 0 ? 16 * (W::UPS - 1) : 0);
            cp_async16((face == 0 ? ws.xlo_ : ws.xhi_) + 16 * W::h(y, z), g, ok);
        }
    } else if constexpr (ASYNC) {
        constexpr int HY = BY + 2, HZ = BZ + 2;
        for (int u = lane; u < 2 * HY * HZ; u += 32) {
            const int face = u / (HY * HZ), v_ = u % (HY * HZ);
            const int y = v_ % HY - 1, z = v_ / HY - 1;
            const bool yin = y >= 0 && y < BY, zin = z >= 0 && z < BZ;
            int r = 1 + face, ys = y, zs = z;
            if (!yin) {
                r = 7 + face + (y == BY ? 2 : 0);
                ys = y < 0 ? BY - 1 : 0;
            } else if (!zin) {
                r = 11 + face + (z == BZ ? 2 : 0);
                zs = z < 0 ? BZ - 1 : 0;
            }
            uint32_t j = 0;
            const bool ok = (yin || zin) &&
                            seg_index(ws.rec[r], (face == 0 ? S::SX - 1 : 0) + S::SX * ys + S::PLANE * zs, j);
            const char *g = reinterpret_cast<const char *>(src + (ok ? j : 0u)) + (face == 0 ? 16 * (W::UPS - 1) : 0);
            cp_async16((face == 0 ? ws.xlo_ : ws.xhi_) + 16 * W::h(y, z), g, ok);
        }
    } else
    // -x / +x faces: single cells (x = BX-1 of the -x brick, x = 0 of the +x
    // brick); for the 19-point stencil also on the halo rows and planes,
    // from the xy-edge (records 7..10) and xz-edge (11..14) neighbours
    {
        constexpr int HY = NP == 19 ? BY + 2 : BY, HZ = NP == 19 ? BZ + 2 : BZ, O = NP == 19 ? 1 : 0;
        // unrolled, so that a lane's loads are all issued before the first
        // of them is waited for
#pragma unroll
        for (int u = lane; u < 2 * HY * HZ; u += 32) {
            const int face = u / (HY * HZ), v_ = u % (HY * HZ);
            const int y = v_ % HY - O, z = v_ / HY - O;
            const bool yin = y >= 0 && y < BY, zin = z >= 0 && z < BZ;
            CT v = czero<CT>();
            if (yin || zin) {  // the y-z corners are read by no stencil
                int r = 1 + face, ys = y, zs = z;
                if (!yin) {
                    r = 7 + face + (y == BY ? 2 : 0);
                    ys = y < 0 ? BY - 1 : 0;
                } else if (!zin) {
                    r = 11 + face + (z == BZ ? 2 : 0);
                    zs = z < 0 ? BZ - 1 : 0;
                }
                uint32_t j;
                if (seg_index(ws.rec[r], (face == 0 ? S::SX - 1 : 0) + S::SX * ys + S::PLANE * zs, j)) {
                    j += face == 0 ? 3 : 0;
                    v = xf(ld1<CG>(src + j), j);
                }
            }
            *(face == 0 ? ws.xm_slot(W::h(y, z)) : ws.xp_slot(W::h(y, z))) = v;
        }
    }
    cp_async_wait_all();
    __syncwarp();
    // stored segments: Laplacian from the tile, then the body.  Opposite
    // neighbours are summed first and the centre term enters once:
    // L = (x- + x+) / hx^2 + (y- + y+) / hy^2 + (z- + z+) / hz^2 - c6 c.
    const R c6 = (R)2 * (ihx2 + ihy2 + ihz2);
    auto segment = [&](int r, const auto &pre) {
        const int e = ws.list[r];
        const int sl = e & 0xff, hrow = e >> 8, hx = sl % S::SX;
        CT c[4], ym[4], yp[4], zm[4], zp[4], L[4];
        ws.get(sl, c);
        ws.get(sl - W::ROW, ym);
        ws.get(sl + W::ROW, yp);
        ws.get(sl - W::PLANE, zm);
        ws.get(sl + W::PLANE, zp);
        const CT xm = hx == 0 ? ws.xm_cell(hrow) : ws.last(sl - 1);
        const CT xp = hx == S::SX - 1 ? ws.xp_cell(hrow) : ws.first(sl + 1);
        if constexpr (NP != 19) {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const CT l = i == 0 ? xm : c[i - 1];
                const CT rr = i == 3 ? xp : c[i + 1];
                L[i] = lapv(rr, l, yp[i], ym[i], zp[i], zm[i], c[i], ihx2, ihy2, ihz2, c6);
            }
        } else {
            // App. B: the 7-point part plus w_ab (edges_ab - 2 faces_ab + 4 c)
            // per plane ab, w_ab = (h_a^2 + h_b^2) / (12 h_a^2 h_b^2)
            // = (1/h_a^2 + 1/h_b^2) / 12.  Each face pair lies in two planes,
            // so the face and centre terms fold into the 7-point form with
            //   x: 1/hx^2 - 2 (wxy + wxz), y: 1/hy^2 - 2 (wxy + wyz),
            //   z: 1/hz^2 - 2 (wxz + wyz), centre: c6 - 4 (wxy + wxz + wyz),
            // and only the three edge sums remain: + wxy exy + wxz exz + wyz eyz.
            const R wxy = (ihx2 + ihy2) / (R)12, wxz = (ihx2 + ihz2) / (R)12, wyz = (ihy2 + ihz2) / (R)12;
            const R ax = ihx2 - (R)2 * (wxy + wxz), ay = ihy2 - (R)2 * (wxy + wyz), az = ihz2 - (R)2 * (wxz + wyz);
            const R c19 = c6 - (R)4 * (wxy + wxz + wyz);
            const int row = sl / S::SX, y = row % W::TY - 1, z = row / W::TY - 1;
            auto left = [&](int s2, int yy, int zz) { return hx == 0 ? ws.xm_cell(W::h(yy, zz)) : ws.last(s2 - 1); };
            auto right = [&](int s2, int yy, int zz) {
                return hx == S::SX - 1 ? ws.xp_cell(W::h(yy, zz)) : ws.first(s2 + 1);
            };
            const CT yml = left(sl - W::ROW, y - 1, z), ymr = right(sl - W::ROW, y - 1, z);
            const CT ypl = left(sl + W::ROW, y + 1, z), ypr = right(sl + W::ROW, y + 1, z);
            const CT zml = left(sl - W::PLANE, y, z - 1), zmr = right(sl - W::PLANE, y, z - 1);
            const CT zpl = left(sl + W::PLANE, y, z + 1), zpr = right(sl + W::PLANE, y, z + 1);
            CT eyz[4], t4[4];
            ws.get(sl - W::ROW - W::PLANE, eyz);
            ws.get(sl + W::ROW - W::PLANE, t4);
#pragma unroll
            for (int i = 0; i < 4; ++i) eyz[i] = vadd(eyz[i], t4[i]);
            ws.get(sl - W::ROW + W::PLANE, t4);
#pragma unroll
            for (int i = 0; i < 4; ++i) eyz[i] = vadd(eyz[i], t4[i]);
            ws.get(sl + W::ROW + W::PLANE, t4);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                eyz[i] = vadd(eyz[i], t4[i]);
                const CT l = i == 0 ? xm : c[i - 1];
                const CT rr = i == 3 ? xp : c[i + 1];
                const CT exy = vadd(vadd(i == 0 ? yml : ym[i - 1], i == 3 ? ymr : ym[i + 1]),
                                    vadd(i == 0 ? ypl : yp[i - 1], i == 3 ? ypr : yp[i + 1]));
                const CT exz = vadd(vadd(i == 0 ? zml : zm[i - 1], i == 3 ? zmr : zm[i + 1]),
                                    vadd(i == 0 ? zpl : zp[i - 1], i == 3 ? zpr : zp[i + 1]));
                L[i] = edgev(lapv(rr, l, yp[i], ym[i], zp[i], zm[i], c[i], ax, ay, az, c19), exy, exz, eyz[i], wxy,
                             wxz, wyz);
            }
        }
        body(R0.off + 4u * (uint32_t)r, pre, c, L);
    };
    // each iteration loads the operands of the next before computing its own
    auto cur = p0;
    for (int r = lane; r < nst; r += 32) {
        decltype(p0) nxt{};
        if (r + 32 < nst) nxt = load(R0.off + 4u * (uint32_t)(r + 32));
        segment(r, cur);
        cur = nxt;
    }
}

// the same without prefetched operands: body(idx, c, L)
template <int BX, int BY, int BZ, bool CG, typename CT, int NP, typename R, typename XF, typename BODY>
__device__ __forceinline__ void brick_apply(WarpSpace<CT, BX, BY, BZ, NP> &ws, const GridView &G, int64_t b,
                                            int64_t next, const CT *src, XF xf, R ihx2, R ihy2, R ihz2, BODY body)
{
    brick_apply<BX, BY, BZ, CG>(ws, G, b, next, src, xf, ihx2, ihy2, ihz2, NoPre(),
                                [&](uint32_t idx, const NoPre::P &, const CT(&c)[4], const CT(&L)[4]) {
                                    body(idx, c, L);
                                });
}

// one-time launch preparation of a stencil kernel: dynamic shared memory
// beyond 48 KiB needs an opt-in; returns resident blocks per SM
template <typename K>
inline int prepare_kernel(K kernel, int threads, size_t smem)
{
    static_assert(sizeof(K) > 0, "");
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int per = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, threads, smem) != cudaSuccess || per < 1) {
        cudaGetLastError();
        per = 1;
    }
    return per;
}

// ------------------------------------------------------------ ramp schedule
struct Ramp {
    const double *clock;  // device time base
    double T;
    int n_knots;
    double knots[GPE_MAX_KNOTS];
};

// s(t): piecewise linear through n_knots values at t_k = k T/(n_knots-1),
// held constant outside [0, T] (linear interpolation between potentials, Sec. V)
__device__ __forceinline__ double ramp_s(const Ramp &r, double t)
{
    if (t <= 0.0) return r.knots[0];
    if (t >= r.T) return r.knots[r.n_knots - 1];
    double u = t / r.T * (double)(r.n_knots - 1);
    int k = (int)floor(u);
    if (k >= r.n_knots - 1) k = r.n_knots - 2;
    double w = u - (double)k;
    return (1.0 - w) * r.knots[k] + w * r.knots[k + 1];
}

template <typename R, typename CT = typename Cx<R>::T>
struct DiagLoad {
    R sc, hg;
    const R *E;
    __device__ __forceinline__ CT apply(CT v, R e) const
    {
        v = scale(v, sc);
        const R f = e >= (R)0 ? e * ((R)1 - hg * norm2(v)) : (R)0;
        return scale(v, f);
    }
    __device__ __forceinline__ CT operator()(CT v, uint32_t idx) const { return apply(v, __ldg(E + idx)); }
    // a whole segment (idx = its first cell): one vector load of E
    __device__ __forceinline__ void seg(CT (&v)[4], uint32_t idx) const
    {
        R e[4];
        ldr4(E + idx, e);
#pragma unroll
        for (int i = 0; i < 4; ++i) v[i] = apply(v[i], e[i]);
    }
};

// deterministic block sum (result valid in thread 0)
__device__ __forceinline__ double block_sum(double x)
{
    __shared__ double sm[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
    __syncthreads();
    if (lane == 0) sm[warp] = x;
    __syncthreads();
    x = 0.0;
    if (warp == 0) {
        x = lane < nw ? sm[lane] : 0.0;
        for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
    }
    return x;
}

// ------------------------------------------------------------ RK4 stages
// Memory-optimised RK4 (App. A, RK4 a* and b*): the stage states are stored
// instead of the k_i, so stage i reads only the state it differentiates (with
// halo) plus own-cell values:
//   stage 0: y2 = y0 + dt/2 f(t, y0)
//   stage 1: y3 = y0 + dt/2 f(t + dt/2, y2),  w = -y0 + y2 + 2 y3
//   stage 2: y4 = y0 + dt   f(t + dt/2, y3)
//   stage 3: y1 = (w + y4)/3 + dt/6 f(t + dt, y4)  (in place of y0)
// with f(t, y) = -i [ -1/2 lap y + (V(t) + g|y|^2) y ]  (Eq. (8)).  The
// partial sum w is formed in stage 1, where y0, y2 and y3 are at hand, in the
// same operation order as the stage-3 combination (-y0 + y2 + 2 y3 + y4)/3:
// stage 3 then reads one state instead of three.  y4 may share y2's buffer
// (y2 has no reader after stage 1).
template <typename R>
struct RkArgs {
    using CT = typename Cx<R>::T;
    CT *y0;
    CT *y2;
    CT *y3;
    CT *y4;
    CT *w;
    const R *V0;
    const R *V1;
    R ihx2, ihy2, ihz2, g, dt;
    Ramp ramp;
    double t_off;  // stage-0 time of this step relative to *ramp.clock
    double dtd;    // dt in FP64 for stage times
};

template <typename R, bool BLEND>
__device__ __forceinline__ R stage_s(const RkArgs<R> &a, int st)
{
    if (!BLEND) return (R)0;
    const double c = (st == 0) ? 0.0 : (st == 3 ? 1.0 : 0.5);
    return (R)ramp_s(a.ramp, *a.ramp.clock + a.t_off + c * a.dtd);
}

// x / 3, correctly rounded, without a division: q = RN(x * RN(1/3)) is within
// one ulp of x/3, the residual r = x - 3q is exact with a fused multiply-add,
// and RN(q + r * RN(1/3)) is the correctly rounded quotient (Markstein's
// theorem on division with a fused multiply-add; Muller et al., Handbook of
// Floating-Point Arithmetic, the section on Newton-Raphson-based division).
__device__ __forceinline__ float div3(float x)
{
    constexpr float t = 1.0f / 3.0f;
    const float q = __fmul_rn(x, t);
    return __fmaf_rn(__fmaf_rn(-3.0f, q, x), t, q);
}
__device__ __forceinline__ double div3(double x)
{
    constexpr double t = 1.0 / 3.0;
    const double q = __dmul_rn(x, t);
    return __fma_rn(__fma_rn(-3.0, q, x), t, q);
}

// One RK4 stage (st = 0..3): operand loads and the per-segment update.  The
// stage is a template argument so that each stage keeps only its own
// prefetched operands in registers.
template <typename R, bool BLEND, bool CG, int st>
struct Rk4Body {
    using CT = typename Cx<R>::T;
    static constexpr int NV = BLEND ? 4 : 1;
    struct P {
        R V0[4], V1[NV];
        CT y[4];  // y0 (stages 1, 2) or w (stage 3)
    };
    const RkArgs<R> &a;
    R s, k;
    CT *yout;
    __device__ __forceinline__ Rk4Body(const RkArgs<R> &a_, R s_)
        : a(a_), s(s_), k(st == 2 ? a_.dt : (st == 3 ? a_.dt / (R)6 : a_.dt / (R)2)),
          yout(st == 0 ? a_.y2 : st == 1 ? a_.y3 : st == 2 ? a_.y4 : a_.y0)
    {
    }
    __device__ __forceinline__ const CT *yin() const { return st == 0 ? a.y0 : st == 1 ? a.y2 : st == 2 ? a.y3 : a.y4; }
    __device__ __forceinline__ P load(uint32_t idx) const
    {
        P p;
        ldr4(a.V0 + idx, p.V0);
        if constexpr (BLEND) ldr4(a.V1 + idx, p.V1);
        if constexpr (st == 1 || st == 2) ld4<CG>(a.y0 + idx, p.y);
        if constexpr (st == 3) ld4<CG>(a.w + idx, p.y);
        return p;
    }
    // the stage's new values o (and, stage 1, the partial sum wv) of the
    // segment with values c, Laplacians L and operands p
    __device__ __forceinline__ void compute(const P &p, const CT (&c)[4], const CT (&L)[4], CT (&o)[4],
                                            CT (&wv)[4]) const
    {
        if constexpr (std::is_same<R, float>::value) {
            // complex64: both parts at once (f32x2), the same operations as the
            // scalar form below
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                if (!(p.V0[i] < (R)INFINITY)) {
                    o[i] = czero<CT>();
                    wv[i] = czero<CT>();
                    continue;
                }
                R V = p.V0[i];
                if constexpr (BLEND) V = ((R)1 - s) * p.V0[i] + s * p.V1[i];
                const R w = V + a.g * (c[i].x * c[i].x + c[i].y * c[i].y);
                const float2 h = fma2(dup2(w), c[i], mul2(dup2(-0.5f), L[i]));   // (hr, hi)
                const float2 hs = make_float2(h.y, h.x);                           // (hi, hr)
                const float2 kk = make_float2(k, -k);                              // f = (hi, -hr)
                if constexpr (st == 0) {
                    o[i] = fma2(kk, hs, c[i]);
                } else if constexpr (st < 3) {
                    o[i] = fma2(kk, hs, p.y[i]);
                    if constexpr (st == 1) wv[i] = fma2(dup2(2.0f), o[i], sub2(c[i], p.y[i]));
                } else {
                    const float2 x = add2(p.y[i], c[i]);
                    const float2 t3 = dup2(1.0f / 3.0f);
                    const float2 q = mul2(x, t3);
                    o[i] = fma2(kk, hs, fma2(fma2(dup2(-3.0f), q, x), t3, q));  // div3 of both parts
                }
            }
            return;
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            if (!(p.V0[i] < (R)INFINITY)) {  // inactive cell of a stored segment
                o[i] = czero<CT>();
                wv[i] = czero<CT>();
                continue;
            }
            R V = p.V0[i];
            if constexpr (BLEND) V = ((R)1 - s) * p.V0[i] + s * p.V1[i];
            const R w = V + a.g * (c[i].x * c[i].x + c[i].y * c[i].y);
            const R hr = (R)(-0.5) * L[i].x + w * c[i].x;
            const R hi = (R)(-0.5) * L[i].y + w * c[i].y;
            // f = -i (hr + i hi) = hi - i hr
            if constexpr (st == 0) {
                o[i].x = c[i].x + k * hi;
                o[i].y = c[i].y - k * hr;
            } else if constexpr (st < 3) {
                o[i].x = p.y[i].x + k * hi;
                o[i].y = p.y[i].y - k * hr;
                if constexpr (st == 1) {
                    wv[i].x = -p.y[i].x + c[i].x + (R)2 * o[i].x;
                    wv[i].y = -p.y[i].y + c[i].y + (R)2 * o[i].y;
                }
            } else {
                o[i].x = div3(p.y[i].x + c[i].x) + k * hi;
                o[i].y = div3(p.y[i].y + c[i].y) - k * hr;
            }
        }
    }
    __device__ __forceinline__ void operator()(uint32_t idx, const P &p, const CT (&c)[4], const CT (&L)[4]) const
    {
        CT o[4], wv[4];
        compute(p, c, L, o, wv);
        if constexpr (st == 1) st4(a.w + idx, wv);
        st4(yout + idx, o);
    }
};

// One RK4 stage on brick b, one warp, lane = segment within each group of 32.
template <typename R, int BX, int BY, int BZ, bool BLEND, bool CG, int st, int NP = 7>
__device__ __forceinline__ void rk4_brick(const RkArgs<R> &a, const GridView &G, int64_t b, int64_t next,
                                          WarpSpace<typename Cx<R>::T, BX, BY, BZ, NP> &ws, R s)
{
    using B = Rk4Body<R, BLEND, CG, st>;
    const B body(a, s);
    brick_apply<BX, BY, BZ, CG>(ws, G, b, next, body.yin(), Identity(), a.ihx2, a.ihy2, a.ihz2,
                                [&](uint32_t idx) { return body.load(idx); }, body);
}

// Programmatic dependent launch: a stage kernel launched with programmatic
// stream serialisation may become resident while the previous stage's last
// blocks still run.  It waits here until that grid has completed and its
// writes are visible, then lets its own dependent launch in turn (once every
// block of this grid has passed this point, so at most two grids share the
// GPU and none waits for a block that cannot become resident).  Without a
// programmatic dependency both instructions return at once.
__device__ __forceinline__ void pdl_enter()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename R, int BX, int BY, int BZ, bool BLEND, int ST, int NP = 7>
__global__ void GPE_BOUNDS_NP(R) k_rk4_staged(const RkArgs<R> a, const GridView G)
{
    pdl_enter();
    constexpr int NW = KernelCfg<R>::NW;
    auto &ws = warp_space<R, BX, BY, BZ, typename Cx<R>::T, NP>();
    const int warp = threadIdx.x >> 5;
    const R s = stage_s<R, BLEND>(a, ST);
    const int64_t stride = (int64_t)gridDim.x * NW;
    for (int64_t b = (int64_t)blockIdx.x * NW + warp; b < G.nb; b += stride)
        rk4_brick<R, BX, BY, BZ, BLEND, false, ST, NP>(a, G, b, b + stride < G.nb ? b + stride : -1, ws, s);
}

// the four stage kernels of one shape, static (BLEND false) or blended, and
// their launch shape
template <typename R, int BX, int BY, int BZ, int NP = 7>
struct Rk4Stages {
    using K = void (*)(RkArgs<R>, GridView);
    static constexpr int NW = KernelCfg<R>::NW;
    static constexpr int THREADS = 32 * NW;
    static constexpr size_t smem() { return smem_bytes<R, BX, BY, BZ, typename Cx<R>::T, NP>(); }
    static K get(bool blend, int st)
    {
        static const K t[2][4] = {
            {k_rk4_staged<R, BX, BY, BZ, false, 0, NP>, k_rk4_staged<R, BX, BY, BZ, false, 1, NP>,
             k_rk4_staged<R, BX, BY, BZ, false, 2, NP>, k_rk4_staged<R, BX, BY, BZ, false, 3, NP>},
            {k_rk4_staged<R, BX, BY, BZ, true, 0, NP>, k_rk4_staged<R, BX, BY, BZ, true, 1, NP>,
             k_rk4_staged<R, BX, BY, BZ, true, 2, NP>, k_rk4_staged<R, BX, BY, BZ, true, 3, NP>}};
        return t[blend ? 1 : 0][st];
    }
};

}  // namespace gpe
