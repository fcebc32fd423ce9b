// Moments and BGK/TRT collision of a fluid cell in the pair form, two
// direction pairs per instruction.
//
// With S_k = a_k + a_opp(k) and D_k = a_k - a_opp(k) (deviation storage:
// a_i = value_i - w_i * ref), a relaxation with rate s on the symmetric part
// and rate a on the antisymmetric part (BGK: s = a) gives the post-collision
// pair a_k = P + M, a_opp(k) = P - M with
//   P = (1 - s)/2 S_k + s E_k,   M = (1 - a)/2 D_k + a O_k,
// E_k, O_k the symmetric / antisymmetric halves of the equilibrium
// deviation of direction k.  The zeroth and first moments follow from the
// same sums: sum_i a_i = a_0 + sum_k S_k, sum_i e_i a_i = sum_k e_k D_k.
//
// In FP32 two pairs share one paired instruction (FADD2 / FMUL2 / FFMA2,
// sm_100 and later); in FP64 the same helpers issue two scalar operations.
// Dot products e_k.u drop the zero components of e_k at compile time.
#pragma once

namespace lbrbc {

__device__ __forceinline__ void add_x2(float a0, float a1, float b0, float b1, float& r0, float& r1) {
    const float2 r = __fadd2_rn(make_float2(a0, a1), make_float2(b0, b1));
    r0 = r.x;
    r1 = r.y;
}
__device__ __forceinline__ void mul_x2(float a0, float a1, float b0, float b1, float& r0, float& r1) {
    const float2 r = __fmul2_rn(make_float2(a0, a1), make_float2(b0, b1));
    r0 = r.x;
    r1 = r.y;
}
__device__ __forceinline__ void fma_x2(float a0, float a1, float b0, float b1, float c0, float c1, float& r0,
                                       float& r1) {
    const float2 r = __ffma2_rn(make_float2(a0, a1), make_float2(b0, b1), make_float2(c0, c1));
    r0 = r.x;
    r1 = r.y;
}
__device__ __forceinline__ void add_x2(double a0, double a1, double b0, double b1, double& r0, double& r1) {
    r0 = a0 + b0;
    r1 = a1 + b1;
}
__device__ __forceinline__ void mul_x2(double a0, double a1, double b0, double b1, double& r0, double& r1) {
    r0 = a0 * b0;
    r1 = a1 * b1;
}
__device__ __forceinline__ void fma_x2(double a0, double a1, double b0, double b1, double c0, double c1, double& r0,
                                       double& r1) {
    r0 = fma(a0, b0, c0);
    r1 = fma(a1, b1, c1);
}

// e_i . u with the zero components of e_i left out (i known at compile time
// after unrolling).
template <class L, typename T>
__device__ __forceinline__ T edot(int i, T ux, T uy, T uz) {
    T r = T(0);
    bool any = false;
    if (L::cx(i) != 0) {
        r = L::cx(i) > 0 ? ux : -ux;
        any = true;
    }
    if (L::cy(i) != 0) {
        r = any ? (L::cy(i) > 0 ? r + uy : r - uy) : (L::cy(i) > 0 ? uy : -uy);
        any = true;
    }
    if (L::cz(i) != 0) r = any ? (L::cz(i) > 0 ? r + uz : r - uz) : (L::cz(i) > 0 ? uz : -uz);
    return r;
}

// Conservation in the storage precision.  The weights rounded to FP32 sum
// to 1 + 1.5e-8 (D3Q19), so a collision written with them creates mass in
// proportion to the local density deviation, and momentum likewise; over
// thousands of steps of a weakly damped flow this drifts by ~1e-5.  Two
// arrangements keep the collision exactly conservative in real arithmetic
// whatever the rounding, leaving only unbiased per-operation rounding:
//  * the rest population takes the remainder of the mass balance,
//    a_0' = (1 - s) a_0 + s (sum a) - 2 sum_k E'_k, which equals the
//    relaxation of a_0 towards its equilibrium when the weights are exact;
//  * the antisymmetric equilibrium uses coefficients c_k = w_k / cs^2 whose
//    sum 2 sum_k c_k e_k e_k = I holds exactly for the rounded values: the
//    diagonal coefficient rounded once, the axis coefficient as 1/2 minus
//    the diagonal ones that share its axis (exact by Sterbenz's lemma).
template <class L>
__host__ __device__ constexpr int diag_per_axis() {
    int n = 0;
    for (int k = 1; k <= L::H; ++k)
        if (L::cx(k) != 0 && L::cx(k) * L::cx(k) + L::cy(k) * L::cy(k) + L::cz(k) * L::cz(k) > 1) ++n;
    return n;
}

// w_k / cs^2 of pair k for a lattice with cs^2 = 1/3 and fixed weights
// (D3Q19, D2Q9), or 1/2 for D3Q7 / D2Q5 (w_k = cs^2 / 2 at any rest
// fraction), in exact-sum form.
template <class L, typename T>
__device__ __forceinline__ T mom_coef(int k) {
    constexpr int nd = diag_per_axis<L>();
    if constexpr (nd == 0) {
        return T(0.5);
    } else {
        const T cd = T(3.0 * L::w(L::H));  // the last pair of the half-split sets is diagonal
        const bool axis = L::cx(k) * L::cx(k) + L::cy(k) * L::cy(k) + L::cz(k) * L::cz(k) == 1;
        return axis ? T(0.5) - T(nd) * cd : cd;
    }
}

// S_k, D_k for k = 1..H (arrays indexed 1..H+1; for odd H the last lane of
// the last instruction repeats pair H).
template <class L, typename T>
__device__ __forceinline__ void pair_sums(const T (&a)[L::Q], T (&S)[L::H + 2], T (&D)[L::H + 2]) {
#pragma unroll
    for (int k = 1; k <= L::H; k += 2) {
        const int k1 = k + 1 <= L::H ? k + 1 : k;
        add_x2(a[k], a[k1], a[L::opp(k)], a[L::opp(k1)], S[k], S[k + 1]);
        fma_x2(a[L::opp(k)], a[L::opp(k1)], T(-1), T(-1), a[k], a[k1], D[k], D[k + 1]);
    }
}

// Post-collision pairs from P, M: a_k = P + M, a_opp(k) = P - M.
template <class L, typename T>
__device__ __forceinline__ void pair_out(T (&a)[L::Q], int k, int k1, T P0, T P1, T M0, T M1) {
    T r0, r1, q0, q1;
    add_x2(P0, P1, M0, M1, r0, r1);
    fma_x2(M0, M1, T(-1), T(-1), P0, P1, q0, q1);
    a[k] = r0;
    a[L::opp(k)] = q0;
    if (k1 != k) {
        a[k1] = r1;
        a[L::opp(k1)] = q1;
    }
}

// Flow cell: moments (rho, u) and collision of the flow populations.
// Equilibrium deviation of direction i: w_i (drho + rho (3 e.u + 4.5 (e.u)^2
// - 1.5 u.u)); E_k = w_k (drho + rho (4.5 (e.u)^2 - 1.5 u.u)),
// O_k = 3 w_k rho e_k.u = 3 w_k e_k.j.
template <class L, typename T>
__device__ __forceinline__ void flow_pairs(T (&f)[L::Q], T& rho, T& ux, T& uy, T& uz, const Phys& p,
                                           const PhysT<T>& q) {
    constexpr int H = L::H;
    T S[H + 2], D[H + 2];
    pair_sums<L, T>(f, S, D);
    T drho = f[0], jx = T(0), jy = T(0), jz = T(0);
#pragma unroll
    for (int k = 1; k <= H; ++k) {
        drho += S[k];
        if (L::cx(k)) jx = L::cx(k) > 0 ? jx + D[k] : jx - D[k];
        if (L::cy(k)) jy = L::cy(k) > 0 ? jy + D[k] : jy - D[k];
        if (L::cz(k)) jz = L::cz(k) > 0 ? jz + D[k] : jz - D[k];
    }
    rho = T(1) + drho;
    const T inv = T(1) / rho;
    ux = jx * inv;
    uy = jy * inv;
    uz = jz * inv;
    const T usq = ux * ux + uy * uy + uz * uz;
    const T s = q.f_sym, a = p.trt_f ? q.f_anti : q.f_sym;
    const T hs = T(0.5) - T(0.5) * s, ha = T(0.5) - T(0.5) * a;
    const T m15 = T(-1.5) * usq;
    T esum = T(0);  // sum of E'_k over the pairs
#pragma unroll
    for (int k = 1; k <= H; k += 2) {
        const int k1 = k + 1 <= H ? k + 1 : k;
        const T e0 = edot<L, T>(k, ux, uy, uz), e1 = edot<L, T>(k1, ux, uy, uz);
        const T j0 = edot<L, T>(k, jx, jy, jz), j1 = edot<L, T>(k1, jx, jy, jz);
        const T sw0 = s * T(L::w(k)), sw1 = s * T(L::w(k1));
        const T aw0 = a * mom_coef<L, T>(k), aw1 = a * mom_coef<L, T>(k1);
        // t = 4.5 (e.u)^2 - 1.5 u.u;  E' = s E = s w (drho + rho t);  O' = a O = a (w / cs^2) e.j
        // (rho u = j: the momentum enters without the rounding of u = j / rho)
        T h0, h1, t0, t1, E0, E1, P0, P1, O0, O1, M0, M1;
        mul_x2(T(4.5) * e0, T(4.5) * e1, e0, e1, h0, h1);
        add_x2(h0, h1, m15, m15, t0, t1);
        fma_x2(rho, rho, t0, t1, drho, drho, t0, t1);
        mul_x2(sw0, sw1, t0, t1, E0, E1);
        esum += k1 != k ? E0 + E1 : E0;
        fma_x2(hs, hs, S[k], S[k + 1], E0, E1, P0, P1);
        mul_x2(aw0, aw1, j0, j1, O0, O1);
        fma_x2(ha, ha, D[k], D[k + 1], O0, O1, M0, M1);
        pair_out<L, T>(f, k, k1, P0, P1, M0, M1);
    }
    // rest population: the remainder of the mass balance
    f[0] = (T(1) - s) * f[0] + (s * drho - T(2) * esum);
}

// Solute cell: collision of the solute populations with concentration C
// (deviation reference cref) and the flow velocity u.  E_k = w_k (C - cref),
// O_k = w_k C e_k.u / cs^2.  Returns C's deviation sum through C.
template <class L, typename T>
__device__ __forceinline__ void solute_pairs(T (&g)[L::Q], T& C, T ux, T uy, T uz, const Phys& p,
                                             const PhysT<T>& q) {
    constexpr int H = L::H;
    T S[H + 2], D[H + 2];
    pair_sums<L, T>(g, S, D);
    T dc = g[0];
#pragma unroll
    for (int k = 1; k <= H; ++k) dc += S[k];
    C = q.cref + dc;
    const T s = p.trt_g ? q.g_sym : q.g_anti, a = q.g_anti;
    const T hs = T(0.5) - T(0.5) * s, ha = T(0.5) - T(0.5) * a;
    T esum = T(0);
#pragma unroll
    for (int k = 1; k <= H; k += 2) {
        const int k1 = k + 1 <= H ? k + 1 : k;
        const T e0 = edot<L, T>(k, ux, uy, uz), e1 = edot<L, T>(k1, ux, uy, uz);
        T E0, E1, P0, P1, O0, O1, M0, M1;
        E0 = s * q.gw[k] * dc;
        E1 = s * q.gw[k1] * dc;
        esum += k1 != k ? E0 + E1 : E0;
        fma_x2(hs, hs, S[k], S[k + 1], E0, E1, P0, P1);
        mul_x2(a * mom_coef<L, T>(k) * C, a * mom_coef<L, T>(k1) * C, e0, e1, O0, O1);
        fma_x2(ha, ha, D[k], D[k + 1], O0, O1, M0, M1);
        pair_out<L, T>(g, k, k1, P0, P1, M0, M1);
    }
    // rest population: the remainder of the mass balance
    g[0] = (T(1) - s) * g[0] + (s * dc - T(2) * esum);
}

}  // namespace lbrbc
