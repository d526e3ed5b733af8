// The D3Q19 lattice of Eq. (1): speeds and weights, population storage
// formats, the pull of the streaming step, the BGK collision with the Guo
// source, the node velocity and the thermal noise. Shared by the library's
// own translation units only.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/lbmd.h"

namespace lbmd {

constexpr int Q = 19;

// D3Q19 speeds in the ABI order (rest, six faces, twelve edges; 2k-1 and 2k
// opposite). Written as constant expressions so unrolled loops fold them.
__host__ __device__ __forceinline__ constexpr int cx(int i) {
    return (i == 1 || i == 7 || i == 9 || i == 11 || i == 13)     ? 1
           : (i == 2 || i == 8 || i == 10 || i == 12 || i == 14) ? -1
                                                                   : 0;
}
__host__ __device__ __forceinline__ constexpr int cy(int i) {
    return (i == 3 || i == 7 || i == 10 || i == 15 || i == 17)    ? 1
           : (i == 4 || i == 8 || i == 9 || i == 16 || i == 18)  ? -1
                                                                   : 0;
}
__host__ __device__ __forceinline__ constexpr int cz(int i) {
    return (i == 5 || i == 11 || i == 14 || i == 15 || i == 18)   ? 1
           : (i == 6 || i == 12 || i == 13 || i == 16 || i == 17) ? -1
                                                                    : 0;
}
__host__ __device__ __forceinline__ constexpr int opp(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }
__host__ __device__ __forceinline__ constexpr float wgt(int i) {
    return i == 0 ? 1.0f / 3.0f : (i <= 6 ? 1.0f / 18.0f : 1.0f / 36.0f);
}

// Storage formats of the populations (delta f = f - w rho0 in every format;
// FP16 scaled by 2^10).
template <int S> struct Store;
template <> struct Store<LBMD_F32> {
    using T = float;
    static __device__ __forceinline__ float ld(const T *p) { return __ldg(p); }
    static __device__ __forceinline__ float ld_plain(const T *p) { return *p; }
    static __device__ __forceinline__ void st(T *p, float v) { __stcs(p, v); }
    static __device__ __forceinline__ void st_plain(T *p, float v) { *p = v; }
    // Stored units (the dense kernels collide in them, see collide_g).
    static constexpr bool kScaled = false;
    static __device__ __forceinline__ float ld_raw(const T *p) { return __ldg(p); }
    static __device__ __forceinline__ void st_raw(T *p, float v) { __stcs(p, v); }
};
// FP16 holds 2^10 delta f: the exact power-of-two scale lifts the small
// deviations of slow flows (down to ~1e-7) out of FP16's subnormal range,
// and |delta f| up to 64 still fits.
constexpr float kF16Scale = 1024.f, kF16Unscale = 1.f / 1024.f;
template <> struct Store<LBMD_F16_SHIFTED> {
    using T = __half;
    static __device__ __forceinline__ float ld(const T *p) { return __half2float(__ldg(p)) * kF16Unscale; }
    static __device__ __forceinline__ float ld_plain(const T *p) { return __half2float(*p) * kF16Unscale; }
    static __device__ __forceinline__ void st(T *p, float v) { __stcs(p, __float2half_rn(v * kF16Scale)); }
    static __device__ __forceinline__ void st_plain(T *p, float v) { *p = __float2half_rn(v * kF16Scale); }
    static constexpr bool kScaled = true;
    static __device__ __forceinline__ float ld_raw(const T *p) { return __half2float(__ldg(p)); }
    static __device__ __forceinline__ void st_raw(T *p, float v) { __stcs(p, __float2half_rn(v)); }
};
template <> struct Store<LBMD_BF16_SHIFTED> {
    using T = __nv_bfloat16;
    static __device__ __forceinline__ float ld(const T *p) { return __bfloat162float(__ldg(p)); }
    static __device__ __forceinline__ float ld_plain(const T *p) { return __bfloat162float(*p); }
    static __device__ __forceinline__ void st(T *p, float v) { __stcs(p, __float2bfloat16_rn(v)); }
    static __device__ __forceinline__ void st_plain(T *p, float v) { *p = __float2bfloat16_rn(v); }
    static constexpr bool kScaled = false;
    static __device__ __forceinline__ float ld_raw(const T *p) { return __bfloat162float(__ldg(p)); }
    static __device__ __forceinline__ void st_raw(T *p, float v) { __stcs(p, __float2bfloat16_rn(v)); }
};

inline size_t store_bytes(int store) { return store == LBMD_F32 ? 4 : 2; }

// Lattice description passed by value to every lattice kernel.
struct Lat {
    int nx, ny, nz;
    size_t N;     // nx*ny*nz, also the plane stride of the SoA populations
    float omega;  // 1/tau
    float rho0;
    int walls;    // z bounce-back walls
    int forcing;  // LBMD_FORCE_*
    float famp;   // body-force amplitude
    int fdir, faxis;
    const float *kshape;  // Kolmogorov wave sin(2 pi c / n_axis), c < n_axis (device table)
    int thermal;          // 1: add the thermal noise xi_i after every collision
    float namp[15];       // noise amplitude of modes 4..18: sqrt(mu (1 - (1 - omega)^2) / b_k)
    unsigned key0, key1;  // noise seed (low, high words)
};

// ---------------------------------------------------------------------------
// Thermal noise of the fluctuating lattice Boltzmann equation: the xi_i of the
// source term S_i = p_i + xi_i of Eq. (1) (Sec. 2.2). After the collision each
// node gets xi_i = w_i sum_{k=4..18} e_k(c_i) a_k n_k: independent standard
// normals n_k on the 15 modes e_k of a moment basis that are not conserved
// (the basis polynomials below are orthogonal under the weights w_i; modes
// 0..3, density and momentum, get none), with a_k = sqrt(mu (1 - (1 -
// omega)^2) / b_k), b_k = sum_i w_i e_k(c_i)^2, mu = rho0 kT / c_s^2: each
// mode then fluctuates with variance mu b_k at rest, as the
// fluctuation-dissipation relation of a relaxation by 1 - omega requires.
// The normals come from the counter-based Philox4x32-10 generator (counter:
// node, block 0..3, step; key: the seed), 23-bit uniforms (m + 1/2) 2^-23,
// and the Box-Muller transform.

// Mode k of the basis at speed i (small integers; constant-folded).
__host__ __device__ __forceinline__ constexpr int emode(int k, int i) {
    const int x = cx(i), y = cy(i), z = cz(i), c2 = x * x + y * y + z * z;
    return k == 0    ? 1
           : k == 1  ? x
           : k == 2  ? y
           : k == 3  ? z
           : k == 4  ? c2 - 1
           : k == 5  ? 3 * x * x - c2
           : k == 6  ? y * y - z * z
           : k == 7  ? x * y
           : k == 8  ? y * z
           : k == 9  ? x * z
           : k == 10 ? (3 * c2 - 5) * x
           : k == 11 ? (3 * c2 - 5) * y
           : k == 12 ? (3 * c2 - 5) * z
           : k == 13 ? (y * y - z * z) * x
           : k == 14 ? (z * z - x * x) * y
           : k == 15 ? (x * x - y * y) * z
           : k == 16 ? 3 * c2 * c2 - 6 * c2 + 1
           : k == 17 ? (2 * c2 - 3) * (3 * x * x - c2)
                     : (2 * c2 - 3) * (y * y - z * z);
}

// Philox4x32-10 block: ten rounds of the two 32x32 -> 64-bit products of the
// published generator, the key advanced by its Weyl constants.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, unsigned k0, unsigned k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const unsigned lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const unsigned lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// Two standard normals from two words (Box-Muller on 23-bit uniforms, exact in FP32).
__device__ __forceinline__ float2 box_muller(unsigned a, unsigned b) {
    const float u1 = ((float)(a >> 9) + 0.5f) * 1.1920928955078125e-7f;  // 2^-23
    const float u2 = ((float)(b >> 9) + 0.5f) * 1.1920928955078125e-7f;
    const float r = sqrtf(-2.f * logf(u1));
    float sn, cs;
    sincospif(2.f * u2, &sn, &cs);
    return make_float2(r * cs, r * sn);
}

// xi_i of one node at one step, scaled by sc (the storage scale of the
// stored deviations the caller adds it to).
__device__ __forceinline__ void node_noise(const Lat &L, unsigned node, unsigned step, float sc, float xi[Q]) {
    float s[16];
#pragma unroll
    for (int call = 0; call < 4; ++call) {
        const uint4 w = philox4x32_10(make_uint4(node, (unsigned)call, step, 0u), L.key0, L.key1);
        const float2 n0 = box_muller(w.x, w.y), n1 = box_muller(w.z, w.w);
        s[4 * call] = n0.x;
        s[4 * call + 1] = n0.y;
        s[4 * call + 2] = n1.x;
        s[4 * call + 3] = n1.y;
    }
#pragma unroll
    for (int k = 0; k < 15; ++k) s[k] *= sc * L.namp[k];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        float acc = 0.f;
#pragma unroll
        for (int k = 4; k < Q; ++k)
            if (emode(k, i) != 0) acc = fmaf((float)emode(k, i), s[k - 4], acc);
        xi[i] = wgt(i) * acc;
    }
}

// Body force g at a node (the Kolmogorov wave from a per-row table, L1-resident).
__device__ __forceinline__ void body_force(const Lat &L, int x, int y, int z, float g[3]) {
    g[0] = g[1] = g[2] = 0.f;
    if (L.forcing == LBMD_FORCE_NONE) return;
    float a = L.famp;
    if (L.forcing == LBMD_FORCE_KOLMOGOROV) {
        int c = L.faxis == 0 ? x : (L.faxis == 1 ? y : z);
        a *= __ldg(L.kshape + c);
    }
    g[L.fdir] = a;
}

// Index of population i pulled into node (x, y, z): the post-collision value
// h_i(x - c_i), or h_opp(i)(x) when x - c_i is behind a z wall (half-way
// bounce-back). Periodic elsewhere.
__device__ __forceinline__ size_t pull_index(const Lat &L, int i, int x, int y, int z, int xm, int xp, int ym,
                                             int yp, int zm, int zp, size_t node) {
    const int sx = cx(i) == 1 ? xm : (cx(i) == -1 ? xp : x);
    const int sy = cy(i) == 1 ? ym : (cy(i) == -1 ? yp : y);
    const int sz = cz(i) == 1 ? zm : (cz(i) == -1 ? zp : z);
    bool wall = false;
    if (L.walls) wall = (cz(i) == 1 && z == 0) || (cz(i) == -1 && z == L.nz - 1);
    return wall ? (size_t)opp(i) * L.N + node : (size_t)i * L.N + ((size_t)sz * L.ny + sy) * L.nx + sx;
}

template <int S>
__device__ __forceinline__ void pull(const typename Store<S>::T *__restrict__ src, const Lat &L, int x, int y,
                                     int z, float f[Q]) {
    const int xm = x == 0 ? L.nx - 1 : x - 1, xp = x == L.nx - 1 ? 0 : x + 1;
    const int ym = y == 0 ? L.ny - 1 : y - 1, yp = y == L.ny - 1 ? 0 : y + 1;
    const int zm = z == 0 ? L.nz - 1 : z - 1, zp = z == L.nz - 1 ? 0 : z + 1;
    const size_t node = ((size_t)z * L.ny + y) * L.nx + x;
#pragma unroll
    for (int i = 0; i < Q; ++i) f[i] = Store<S>::ld(src + pull_index(L, i, x, y, z, xm, xp, ym, yp, zm, zp, node));
}

// BGK collision with the Guo source on deviations (Eq. 1, standard minus
// sign): f_i <- f_i - omega (f_i - f_eq_i) + (1 - omega/2) w_i [3(c_i - u) +
// 9 (c_i.u) c_i].F with u = (sum f c + F/2)/rho; every value shifted by
// w_i rho0. Returns rho.
__device__ __forceinline__ float collide(const Lat &L, float f[Q], const float F[3]) {
    float drho = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        drho += f[i];
        if (cx(i)) jx += cx(i) * f[i];
        if (cy(i)) jy += cy(i) * f[i];
        if (cz(i)) jz += cz(i) * f[i];
    }
    const float rho = L.rho0 + drho;
    const float inv = 1.f / rho;
    const float ux = (jx + 0.5f * F[0]) * inv, uy = (jy + 0.5f * F[1]) * inv, uz = (jz + 0.5f * F[2]) * inv;
    const float usq = ux * ux + uy * uy + uz * uz;
    const float uF = ux * F[0] + uy * F[1] + uz * F[2];
    const float om = L.omega, src = 1.f - 0.5f * om;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const float cu = cx(i) * ux + cy(i) * uy + cz(i) * uz;
        const float cF = cx(i) * F[0] + cy(i) * F[1] + cz(i) * F[2];
        const float feq = wgt(i) * (drho + rho * (3.f * cu + 4.5f * cu * cu - 1.5f * usq));
        const float S = src * wgt(i) * (3.f * (cF - uF) + 9.f * cu * cF);
        f[i] = f[i] - om * (f[i] - feq) + S;
    }
    return rho;
}

// Amplitude a of the body force g = a e_fdir at a node (0 without forcing).
__device__ __forceinline__ float body_amp(const Lat &L, int x, int y, int z) {
    if (L.forcing == LBMD_FORCE_NONE) return 0.f;
    float a = L.famp;
    if (L.forcing == LBMD_FORCE_KOLMOGOROV) {
        const int c = L.faxis == 0 ? x : (L.faxis == 1 ? y : z);
        a *= __ldg(L.kshape + c);
    }
    return a;
}

// BGK collision + Guo source of one node whose force is the body force
// g = ga e_FD (FD = -1: no force), specialised at compile time on FD so only
// the speeds with a component along FD carry force terms. f holds SC times
// the pulled deviations delta f (SC = 2^10 for FP16 storage, else 1) and
// receives SC times the post-collision deviations. Speeds are taken with
// their opposites: with cu = c_i.u and cF = c_i.F,
//   new f_i = (1 - omega) f_i + SC w_i (E + O),  new f_opp = (1 - omega) f_opp + SC w_i (E - O),
//   E = A0 + cu (9/2 omega rho cu + 9 s cF),  O = 3 omega rho cu + 3 s cF,
//   A0 = omega (drho - 3/2 rho u.u) - 3 s u.F,  s = 1 - omega/2,
// E the even and O the odd part of the equilibrium and the Guo source, and
// SC w_i folded into per-class constants (faces 1/18, edges 1/36).
// Returns rho.
template <int FD, bool SCALED>
__device__ __forceinline__ float collide_g(const Lat &L, float f[Q], float ga) {
    constexpr float sc = SCALED ? kF16Scale : 1.f, isc = SCALED ? kF16Unscale : 1.f;
    float sp[9], dp[9];
#pragma unroll
    for (int p = 0; p < 9; ++p) {
        sp[p] = f[2 * p + 1] + f[2 * p + 2];
        dp[p] = f[2 * p + 1] - f[2 * p + 2];
    }
    float drho = f[0], jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
    for (int p = 0; p < 9; ++p) {
        drho += sp[p];
        if (cx(2 * p + 1)) jx += cx(2 * p + 1) * dp[p];
        if (cy(2 * p + 1)) jy += cy(2 * p + 1) * dp[p];
        if (cz(2 * p + 1)) jz += cz(2 * p + 1) * dp[p];
    }
    if (SCALED) {
        drho *= isc;
        jx *= isc;
        jy *= isc;
        jz *= isc;
    }
    const float rho = L.rho0 + drho;
    const float inv = 1.f / rho;
    if (FD == 0) jx += 0.5f * ga;
    if (FD == 1) jy += 0.5f * ga;
    if (FD == 2) jz += 0.5f * ga;
    const float ux = jx * inv, uy = jy * inv, uz = jz * inv;
    const float usq = ux * ux + uy * uy + uz * uz;
    const float om = L.omega, s = 1.f - 0.5f * om, keep = 1.f - om;
    const float uF = FD == 0 ? ux * ga : (FD == 1 ? uy * ga : (FD == 2 ? uz * ga : 0.f));
    const float A0 = FD >= 0 ? om * (drho - 1.5f * rho * usq) - 3.f * s * uF : om * (drho - 1.5f * rho * usq);
    const float orho = om * rho;
    constexpr float wf = sc / 18.f, we = sc / 36.f;
    const float A0f = wf * A0, A0e = we * A0;
    const float k45f = (4.5f * wf) * orho, k45e = (4.5f * we) * orho;
    const float k3f = (3.f * wf) * orho, k3e = (3.f * we) * orho;
    const float sga = s * ga;
    const float a9f = (9.f * wf) * sga, a9e = (9.f * we) * sga;
    const float a3f = (3.f * wf) * sga, a3e = (3.f * we) * sga;
    // E + O = (A0 + cF a3) + cu (k45 cu + cF a9 + k3), E - O likewise with -k3
    // and -a3: per class and sign of c_i.F, two nested FMAs per result.
    const float Ppf = a9f + k3f, Pmf = a9f - k3f, Qpf = A0f + a3f, Qmf = A0f - a3f;
    const float Ppe = a9e + k3e, Pme = a9e - k3e, Qpe = A0e + a3e, Qme = A0e - a3e;
    f[0] = keep * f[0] + (sc / 3.f) * A0;
#pragma unroll
    for (int i = 1; i < Q; i += 2) {
        const bool face = i <= 6;
        const float cu = cx(i) * ux + cy(i) * uy + cz(i) * uz;
        const int cf = FD == 0 ? cx(i) : (FD == 1 ? cy(i) : (FD == 2 ? cz(i) : 0));
        const float k45 = face ? k45f : k45e;
        float inP, inM, outP, outM;  // E + O = fma(cu, fma(k45, cu, inP), outP), E - O with inM, outM
        if (cf == 0) {
            inP = face ? k3f : k3e;
            inM = -inP;
            outP = outM = face ? A0f : A0e;
        } else if (cf > 0) {
            inP = face ? Ppf : Ppe;
            inM = face ? Pmf : Pme;
            outP = face ? Qpf : Qpe;
            outM = face ? Qmf : Qme;
        } else {
            inP = -(face ? Pmf : Pme);
            inM = -(face ? Ppf : Ppe);
            outP = face ? Qmf : Qme;
            outM = face ? Qpf : Qpe;
        }
        const float EpO = fmaf(cu, fmaf(k45, cu, inP), outP);
        const float EmO = fmaf(cu, fmaf(k45, cu, inM), outM);
        f[i] = fmaf(keep, f[i], EpO);
        f[i + 1] = fmaf(keep, f[i + 1], EmO);
    }
    return rho;
}

// Packed FP32x2 arithmetic (two independent IEEE FP32 lanes per instruction).
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, f2(-1.f), a); }  // a - b, one rounding
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }

// collide_g for two nodes at once that share the body force (the node pairs
// of the 16-bit kernel): the same operations, each on a pair of FP32 lanes
// with the packed FP32x2 instructions, so every lane rounds exactly as one
// scalar operation would. Returns both densities.
template <int FD, bool SCALED>
__device__ __forceinline__ float2 collide_g2(const Lat &L, float2 f[Q], float ga) {
    constexpr float sc = SCALED ? kF16Scale : 1.f, isc = SCALED ? kF16Unscale : 1.f;
    float2 sp[9], dp[9];
#pragma unroll
    for (int p = 0; p < 9; ++p) {
        sp[p] = add2(f[2 * p + 1], f[2 * p + 2]);
        dp[p] = sub2(f[2 * p + 1], f[2 * p + 2]);
    }
    float2 drho = f[0], jx = f2(0.f), jy = f2(0.f), jz = f2(0.f);
#pragma unroll
    for (int p = 0; p < 9; ++p) {
        drho = add2(drho, sp[p]);
        if (cx(2 * p + 1)) jx = cx(2 * p + 1) > 0 ? add2(jx, dp[p]) : sub2(jx, dp[p]);
        if (cy(2 * p + 1)) jy = cy(2 * p + 1) > 0 ? add2(jy, dp[p]) : sub2(jy, dp[p]);
        if (cz(2 * p + 1)) jz = cz(2 * p + 1) > 0 ? add2(jz, dp[p]) : sub2(jz, dp[p]);
    }
    if (SCALED) {
        drho = mul2(drho, f2(isc));
        jx = mul2(jx, f2(isc));
        jy = mul2(jy, f2(isc));
        jz = mul2(jz, f2(isc));
    }
    const float2 rho = add2(f2(L.rho0), drho);
    const float2 inv = make_float2(1.f / rho.x, 1.f / rho.y);
    if (FD == 0) jx = add2(jx, f2(0.5f * ga));
    if (FD == 1) jy = add2(jy, f2(0.5f * ga));
    if (FD == 2) jz = add2(jz, f2(0.5f * ga));
    const float2 ux = mul2(jx, inv), uy = mul2(jy, inv), uz = mul2(jz, inv);
    const float2 usq = fma2(uz, uz, fma2(uy, uy, mul2(ux, ux)));
    const float om = L.omega, s = 1.f - 0.5f * om, keep = 1.f - om;
    float2 A0 = mul2(f2(om), fma2(mul2(f2(-1.5f), rho), usq, drho));
    if (FD >= 0) {
        const float2 uF = mul2(FD == 0 ? ux : (FD == 1 ? uy : uz), f2(ga));
        A0 = fma2(f2(-3.f * s), uF, A0);
    }
    const float2 orho = mul2(f2(om), rho);
    constexpr float wf = sc / 18.f, we = sc / 36.f;
    const float2 A0f = mul2(f2(wf), A0), A0e = mul2(f2(we), A0);
    const float2 k45f = mul2(f2(4.5f * wf), orho), k45e = mul2(f2(4.5f * we), orho);
    const float2 k3f = mul2(f2(3.f * wf), orho), k3e = mul2(f2(3.f * we), orho);
    const float sga = s * ga;
    const float2 a9f = f2((9.f * wf) * sga), a9e = f2((9.f * we) * sga);
    const float2 a3f = f2((3.f * wf) * sga), a3e = f2((3.f * we) * sga);
    const float2 Ppf = add2(a9f, k3f), Pmf = sub2(a9f, k3f), Qpf = add2(A0f, a3f), Qmf = sub2(A0f, a3f);
    const float2 Ppe = add2(a9e, k3e), Pme = sub2(a9e, k3e), Qpe = add2(A0e, a3e), Qme = sub2(A0e, a3e);
    f[0] = fma2(f2(keep), f[0], mul2(f2(sc / 3.f), A0));
#pragma unroll
    for (int i = 1; i < Q; i += 2) {
        const bool face = i <= 6;
        float2 cu = f2(0.f);
        bool first = true;
        if (cx(i)) {
            cu = cx(i) > 0 ? ux : neg2(ux);
            first = false;
        }
        if (cy(i)) {
            cu = first ? (cy(i) > 0 ? uy : neg2(uy)) : (cy(i) > 0 ? add2(cu, uy) : sub2(cu, uy));
            first = false;
        }
        if (cz(i)) cu = first ? (cz(i) > 0 ? uz : neg2(uz)) : (cz(i) > 0 ? add2(cu, uz) : sub2(cu, uz));
        const int cf = FD == 0 ? cx(i) : (FD == 1 ? cy(i) : (FD == 2 ? cz(i) : 0));
        const float2 k45 = face ? k45f : k45e;
        float2 inP, inM, outP, outM;  // E + O = fma(cu, fma(k45, cu, inP), outP), E - O with inM, outM
        if (cf == 0) {
            inP = face ? k3f : k3e;
            inM = neg2(inP);
            outP = outM = face ? A0f : A0e;
        } else if (cf > 0) {
            inP = face ? Ppf : Ppe;
            inM = face ? Pmf : Pme;
            outP = face ? Qpf : Qpe;
            outM = face ? Qmf : Qme;
        } else {
            inP = neg2(face ? Pmf : Pme);
            inM = neg2(face ? Ppf : Ppe);
            outP = face ? Qmf : Qme;
            outM = face ? Qpf : Qpe;
        }
        const float2 EpO = fma2(cu, fma2(k45, cu, inP), outP);
        const float2 EmO = fma2(cu, fma2(k45, cu, inM), outM);
        f[i] = fma2(f2(keep), f[i], EpO);
        f[i + 1] = fma2(f2(keep), f[i + 1], EmO);
    }
    return rho;
}

// Velocity u = (sum f c + g/2)/rho of a node from its pulled deviations.
__device__ __forceinline__ float node_velocity(const Lat &L, const float f[Q], const float g[3], float u[3]) {
    float drho = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        drho += f[i];
        if (cx(i)) jx += cx(i) * f[i];
        if (cy(i)) jy += cy(i) * f[i];
        if (cz(i)) jz += cz(i) * f[i];
    }
    const float rho = L.rho0 + drho;
    const float inv = 1.f / rho;
    u[0] = (jx + 0.5f * g[0]) * inv;
    u[1] = (jy + 0.5f * g[1]) * inv;
    u[2] = (jz + 0.5f * g[2]) * inv;
    return rho;
}

// Device error flags (bit mask), raised with atomicOr, read by the host.
enum : int { FLAG_NONFINITE = 1, FLAG_CELL = 2, FLAG_WALL = 4, FLAG_TOUCHED = 8 };

// Device-resident step state, updated by the last kernel of each step.
struct DevState {
    int step;        // coupled steps done since the last set_state
    int n_touched;   // unique nodes claimed by atoms this step
    int flags;       // FLAG_* bits
    unsigned ticket; // last-block detection of the fix-up kernel
    int nl_flag[3];  // neighbour-list rebuild requests, by generation mod 3
};

// Launch shape of the one-thread-per-node kernels: rows of x in the block's
// x dimension (a multiple of 32, at most 256 threads), rows of y stacked.
inline dim3 node_block(const Lat &L) {
    int bx = ((L.nx + 31) / 32) * 32;
    if (bx > 256) bx = 256;
    int by = 256 / bx;
    if (by > L.ny) by = L.ny;
    return dim3(bx, by, 1);
}

inline dim3 node_grid(const Lat &L, dim3 b) { return dim3((L.nx + b.x - 1) / b.x, (L.ny + b.y - 1) / b.y, L.nz); }

// Runs KERNEL_CALL with T and SV bound to the storage format's element type
// and tag.
#define LBMD_DISPATCH(store, KERNEL_CALL)                                                                           \
    switch (store) {                                                                                                \
    case LBMD_F32: {                                                                                                \
        using T = float;                                                                                            \
        constexpr int SV = LBMD_F32;                                                                                \
        KERNEL_CALL;                                                                                                \
    } break;                                                                                                        \
    case LBMD_F16_SHIFTED: {                                                                                        \
        using T = __half;                                                                                           \
        constexpr int SV = LBMD_F16_SHIFTED;                                                                        \
        KERNEL_CALL;                                                                                                \
    } break;                                                                                                        \
    default: {                                                                                                      \
        using T = __nv_bfloat16;                                                                                    \
        constexpr int SV = LBMD_BF16_SHIFTED;                                                                       \
        KERNEL_CALL;                                                                                                \
    }                                                                                                               \
    }

// Runs BODY with FDV bound at compile time to the body-force direction
// (-1 without forcing) and THV to the thermal-noise switch.
#define LBMD_FD_DISPATCH1(L, BODY)                                         \
    switch ((L).forcing == LBMD_FORCE_NONE ? -1 : (L).fdir) {             \
        case -1: { constexpr int FDV = -1; BODY; } break;                  \
        case 0: { constexpr int FDV = 0; BODY; } break;                    \
        case 1: { constexpr int FDV = 1; BODY; } break;                    \
        default: { constexpr int FDV = 2; BODY; } break;                   \
    }
#define LBMD_FD_DISPATCH(L, BODY)                                          \
    if ((L).thermal) {                                                     \
        constexpr bool THV = true;                                         \
        LBMD_FD_DISPATCH1(L, BODY)                                         \
    } else {                                                               \
        constexpr bool THV = false;                                        \
        LBMD_FD_DISPATCH1(L, BODY)                                         \
    }

}  // namespace lbmd
