// Discrete adjoint of the solute part of the coupled step, for the gradient
// of the reacted mass J = sum over steps and reactive links of m_l (the
// ledger of Eq. solidFractionUpdate's reading) with respect to k_r (scalar
// or per voxel) and c_eq.  Phase change is frozen (no events), so one step
// is affine in the post-collision solute populations g*:
//   pull (halfway bounce-back, open-boundary rules)  ->  h
//   Eq. general_RBC on the links of wet boundary cells  ->  h'
//   J += sum_links (h'_o - h_o)
//   BGK / TRT collision with the flow velocity of that step  ->  g*.
// The flow does not depend on k_r or c_eq, so its velocity is a recorded
// input.  The kernels below apply the transpose of each stage in reverse
// order: collision, ledger + RBC (with the parameter gradients), streaming.
// Adjoint populations are stored in a plain layout lam[i][cell] (not the AA
// layout), in the storage precision; gradient accumulators are FP64.
#pragma once

namespace lbrbc {

// mu = M^T lam for the collision M (BGK: s = a = omega; TRT: s relaxes the
// symmetric, a the antisymmetric part); e_i = w_i (1 + e_i.u / cs^2).
template <class L, typename T>
__device__ __forceinline__ void collide_transpose(const T (&lam)[L::Q], T (&mu)[L::Q], T ux, T uy, T uz,
                                                  const Phys& p, const PhysT<T>& q) {
    const T s = p.trt_g ? q.g_sym : q.g_anti, a = q.g_anti;
    T pv[L::Q];
    pv[0] = s * lam[0];
#pragma unroll
    for (int i = 1; i <= L::H; ++i) {
        const int j = L::opp(i);
        const T sp = T(0.5) * (lam[i] + lam[j]), sm = T(0.5) * (lam[i] - lam[j]);
        pv[i] = s * sp + a * sm;
        pv[j] = s * sp - a * sm;
    }
    T dot = T(0);
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        const T eu = T(L::cx(i)) * ux + T(L::cy(i)) * uy + T(L::cz(i)) * uz;
        dot += q.gw[i] * (T(1) + eu * q.ics2) * pv[i];
    }
#pragma unroll
    for (int i = 0; i < L::Q; ++i) mu[i] = lam[i] - pv[i] + dot;
}

// Fluid cells: nu = M^T lam (no boundary condition acts on them).
template <typename T, class LG>
__global__ void __launch_bounds__(FLUID_BLOCK) k_adj_fluid(const Dev<T> a, const Phys p, const PhysT<T> q,
                                                        const T* __restrict__ lam, T* __restrict__ nu,
                                                        const float* __restrict__ ut) {
    const Geo& g = a.geo;
    const long long NP = g.NP;
    {
        const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y, z = blockIdx.z;
        if (x >= g.nx) return;
        const long long id = g.idx(x, y, z);
        if ((a.nw[id] & 3u) != CLS_FLUID) return;
        T l[LG::Q], m[LG::Q];
#pragma unroll
        for (int i = 0; i < LG::Q; ++i) l[i] = lam[i * NP + id];
        const T ux = ut ? T(ut[3 * id]) : T(0), uy = ut ? T(ut[3 * id + 1]) : T(0), uz = ut ? T(ut[3 * id + 2]) : T(0);
        collide_transpose<LG, T>(l, m, ux, uy, uz, p, q);
#pragma unroll
        for (int i = 0; i < LG::Q; ++i) nu[i * NP + id] = m[i];
    }
}

// Wet boundary cells: collision transpose (u = 0), ledger and RBC transpose,
// and the parameter gradients of this step.  gprev is this step's tape of
// the streamed h_obar of every reactive link (deviation storage).
// dk: per-cell dJ/dk_r (FP64, may be null); part: per-block partials of the
// scalar dJ/dk_r and dJ/dc_eq (FP64, accumulated over steps).
template <typename T, class LG>
__global__ void __launch_bounds__(LIST_BLOCK, 4) k_adj_bound(const Dev<T> a, const Phys p, const PhysT<T> q,
                                                         const T* __restrict__ lam, T* __restrict__ nu,
                                                         const T* __restrict__ gprev, double* __restrict__ dk,
                                                         double* __restrict__ part) {
    constexpr int Q = LG::Q;
    const Geo& g = a.geo;
    const long long NP = g.NP;
    const int n = *a.nb;
    double gk = 0.0, gc = 0.0;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
        int x, y, z;
        unpack_xyz(a.b_xyz[e], x, y, z);
        const long long b = g.idx(x, y, z);
        const uint32_t bw = a.b_word[e];
        const bool dir = (bw & BW_DIRICHLET) != 0u;
        T l[Q], m[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) l[i] = lam[i * NP + b];
        collide_transpose<LG, T>(l, m, T(0), T(0), T(0), p, q);
        const double kr = a.b_krate ? a.b_krate[e] : p.k_r;
        double cell_k = 0.0;
        T out[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) out[i] = m[i];
#pragma unroll
        for (int o = 1; o < Q; ++o) {
            if (!((bw >> (BW_LINK + o - 1)) & 1u)) continue;
            out[o] = dir ? T(0) : T(-1);  // the replaced h_o enters J only as -h_o (reactive links)
        }
#pragma unroll
        for (int o = 1; o < Q; ++o) {
            if (!((bw >> (BW_LINK + o - 1)) & 1u)) continue;
            const int ob = LG::opp(o);
            if (dir) {
                out[ob] += -m[o];
                continue;
            }
            const T mo = m[o] + T(1);  // dJ/dh'_o: future through the collision, plus the ledger
            if constexpr (sizeof(T) == 4) {
                // FP32 storage: the link terms in FP32 (GB300's FP64 rate is a
                // small fraction of its FP32 rate), in the deviation form of the
                // forward rule; each term is added to the FP64 sums once
                const T kap = a.b_kappa[(long long)(o - 1) * a.cap_b + e];
                T dkdkr = T(0);
                bool inf32 = false;
                if (p.scheme == 0) dkdkr = q.gamma * kap * q.ics2;
                else if (p.scheme == 1) dkdkr = kap * q.ics2;
                else if (p.scheme == 2) {
                    if (kap > T(0)) dkdkr = q.gamma * q.ics2 / kap;
                    else inf32 = true;
                } else inf32 = true;
                if (kr == 0.0) {
                    out[ob] += mo;
                    continue;
                }
                const T w2 = T(2) * q.gw[o];
                if (inf32) {
                    out[ob] += -mo;
                    gc += (double)(mo * w2);
                    continue;
                }
                const T k = dkdkr * T(kr);
                const T ik = T(1) / (T(1) + k);
                out[ob] += (T(1) - k) * ik * mo;
                // dh'_o/dk = (2 w (c_eq - c_ref) - 2 h_obar') / (1 + k)^2
                const T dh = (w2 * q.c_eq_d - T(2) * gprev[(long long)(o - 1) * a.cap_b + e]) * ik * ik;
                cell_k += (double)(mo * dh * dkdkr);
                gc += (double)(mo * k * ik * w2);
                continue;
            }
            const double kap = (double)a.b_kappa[(long long)(o - 1) * a.cap_b + e];
            double dkdkr = 0.0;
            bool inf = false;
            if (p.scheme == 0) dkdkr = p.gamma * kap / p.gcs2;
            else if (p.scheme == 1) dkdkr = kap / p.gcs2;
            else if (p.scheme == 2) {
                if (kap > 0.0) dkdkr = p.gamma / (p.gcs2 * kap);
                else inf = true;
            } else inf = true;
            if (kr == 0.0) {  // inert cell: beta = 1, no dependence on k_r or c_eq
                out[ob] += mo;
                continue;
            }
            const double k = dkdkr * kr;
            const double w = (double)q.gw[o];
            if (inf) {
                out[ob] += -mo;  // anti-bounce-back limit: beta = -1, no k dependence
                gc += (double)mo * 2.0 * w;
                continue;
            }
            const double ik = 1.0 / (1.0 + k);
            out[ob] += T((1.0 - k) * ik) * mo;
            const double hob = (double)gprev[(long long)(o - 1) * a.cap_b + e] + w * p.cref;
            // dh'_o/dk = (2 w c_eq - 2 h_obar) / (1 + k)^2, dk/dk_r = dkdkr
            const double dh = (2.0 * w * p.c_eq - 2.0 * hob) * ik * ik;
            cell_k += (double)mo * dh * dkdkr;
            gc += (double)mo * k * ik * 2.0 * w;
        }
        gk += cell_k;
        if (dk) dk[b] += cell_k;
#pragma unroll
        for (int i = 0; i < Q; ++i) nu[i * NP + b] = out[i];
    }
    gk = warp_sum(gk);
    gc = warp_sum(gc);
    __shared__ double red[2][LIST_BLOCK / 32];
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = gk;
        red[1][threadIdx.x >> 5] = gc;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s0 = 0.0, s1 = 0.0;
        for (int k = 0; k < LIST_BLOCK / 32; ++k) {
            s0 += red[0][k];
            s1 += red[1][k];
        }
        part[2 * blockIdx.x] += s0;
        part[2 * blockIdx.x + 1] += s1;
    }
}

// Streaming transpose (gather form): lam_out_i(y) collects every use of
// g*_i(y) in the step: the pull of y + e_i, or y's own bounce-back /
// open-boundary rule when y + e_i is inactive or outside, and the outlet's
// dependence on y's previous concentration.
template <typename T, class LG>
__global__ void __launch_bounds__(FLUID_BLOCK) k_adj_stream(const Dev<T> a, const Phys p, const PhysT<T> q,
                                                         const T* __restrict__ nu, T* __restrict__ lam_out) {
    const Geo& g = a.geo;
    const long long NP = g.NP;
    {
        const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y, z = blockIdx.z;
        if (x >= g.nx) return;
        const long long id = g.idx(x, y, z);
        const uint32_t cls = a.nw[id] & 3u;
        if (cls == CLS_SOLID) return;
        const bool fluid = cls == CLS_FLUID;
        const bool outlet = fluid && g.open_x && x == g.nx - 1;
        T res[LG::Q];
        T sout = T(0);
#pragma unroll
        for (int i = 0; i < LG::Q; ++i) {
            int xx = x + LG::cx(i), yy = y + LG::cy(i), zz = z + LG::cz(i);
            const bool out_in = g.open_x && xx < 0, out_out = g.open_x && xx >= g.nx;
            const bool inside = !out_in && !out_out && wrap_inside(g, xx, yy, zz);
            const long long nb = inside ? g.idx(xx, yy, zz) : -1;
            const bool active = inside && (a.nw[nb] & 3u) != CLS_SOLID;
            const int ib = LG::opp(i);
            if (i == 0) res[0] = nu[id];
            else if (active) res[i] = nu[(long long)i * NP + nb];
            else if (fluid && out_in) res[i] = -nu[(long long)ib * NP + id];
            else if (fluid && out_out) {
                res[i] = -nu[(long long)ib * NP + id];
                sout += T(2) * q.gw[ib] * nu[(long long)ib * NP + id];
            } else res[i] = nu[(long long)ib * NP + id];
        }
        (void)outlet;
#pragma unroll
        for (int i = 0; i < LG::Q; ++i) lam_out[(long long)i * NP + id] = res[i] + sout;
    }
}

}  // namespace lbrbc
