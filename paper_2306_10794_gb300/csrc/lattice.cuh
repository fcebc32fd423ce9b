// Velocity sets of the device path.  Directions are stored "half split":
// 0 is rest, 1..H the directions with a positive leading component and
// H+1..2H their opposites in the same order, so opp(i) = i +/- H and the TRT
// pairs (i, opp(i)) are found at compile time.  The flow sets carry their
// standard weights (cs^2 = 1/3); the solute weights of D2Q5 / D3Q7 depend on
// the rest fraction J0 (Eqs. RestFraction, RestFractionCs2) and are passed at
// run time, D2Q9 used as a solute lattice keeps its fixed weights.
#pragma once

namespace lbrbc {

struct NoFlow {
    static constexpr int Q = 0, H = 0, DIM = 0;
    __host__ __device__ static constexpr int cx(int) { return 0; }
    __host__ __device__ static constexpr int cy(int) { return 0; }
    __host__ __device__ static constexpr int cz(int) { return 0; }
    __host__ __device__ static constexpr int opp(int i) { return i; }
    __host__ __device__ static constexpr double w(int) { return 0.0; }
};

struct D3Q19 {
    static constexpr int Q = 19, H = 9, DIM = 3;
    __host__ __device__ static constexpr int cx(int i) {
        constexpr int t[19] = {0, 1, 0, 0, 1, 1, 1, 1, 0, 0, -1, 0, 0, -1, -1, -1, -1, 0, 0};
        return t[i];
    }
    __host__ __device__ static constexpr int cy(int i) {
        constexpr int t[19] = {0, 0, 1, 0, 1, -1, 0, 0, 1, 1, 0, -1, 0, -1, 1, 0, 0, -1, -1};
        return t[i];
    }
    __host__ __device__ static constexpr int cz(int i) {
        constexpr int t[19] = {0, 0, 0, 1, 0, 0, 1, -1, 1, -1, 0, 0, -1, 0, 0, -1, 1, -1, 1};
        return t[i];
    }
    __host__ __device__ static constexpr int opp(int i) { return i == 0 ? 0 : (i <= H ? i + H : i - H); }
    __host__ __device__ static constexpr double w(int i) {
        return i == 0 ? 1.0 / 3.0 : (cx(i) * cx(i) + cy(i) * cy(i) + cz(i) * cz(i) == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
    }
};

struct D3Q7 {
    static constexpr int Q = 7, H = 3, DIM = 3;
    __host__ __device__ static constexpr int cx(int i) {
        constexpr int t[7] = {0, 1, 0, 0, -1, 0, 0};
        return t[i];
    }
    __host__ __device__ static constexpr int cy(int i) {
        constexpr int t[7] = {0, 0, 1, 0, 0, -1, 0};
        return t[i];
    }
    __host__ __device__ static constexpr int cz(int i) {
        constexpr int t[7] = {0, 0, 0, 1, 0, 0, -1};
        return t[i];
    }
    __host__ __device__ static constexpr int opp(int i) { return i == 0 ? 0 : (i <= H ? i + H : i - H); }
    __host__ __device__ static constexpr double w(int i) { return i == 0 ? 0.25 : 0.125; }
};

struct D2Q9 {
    static constexpr int Q = 9, H = 4, DIM = 2;
    __host__ __device__ static constexpr int cx(int i) {
        constexpr int t[9] = {0, 1, 0, 1, 1, -1, 0, -1, -1};
        return t[i];
    }
    __host__ __device__ static constexpr int cy(int i) {
        constexpr int t[9] = {0, 0, 1, 1, -1, 0, -1, -1, 1};
        return t[i];
    }
    __host__ __device__ static constexpr int cz(int) { return 0; }
    __host__ __device__ static constexpr int opp(int i) { return i == 0 ? 0 : (i <= H ? i + H : i - H); }
    __host__ __device__ static constexpr double w(int i) {
        return i == 0 ? 4.0 / 9.0 : (cx(i) * cx(i) + cy(i) * cy(i) == 1 ? 1.0 / 9.0 : 1.0 / 36.0);
    }
};

struct D2Q5 {
    static constexpr int Q = 5, H = 2, DIM = 2;
    __host__ __device__ static constexpr int cx(int i) {
        constexpr int t[5] = {0, 1, 0, -1, 0};
        return t[i];
    }
    __host__ __device__ static constexpr int cy(int i) {
        constexpr int t[5] = {0, 0, 1, 0, -1};
        return t[i];
    }
    __host__ __device__ static constexpr int cz(int) { return 0; }
    __host__ __device__ static constexpr int opp(int i) { return i == 0 ? 0 : (i <= H ? i + H : i - H); }
    __host__ __device__ static constexpr double w(int i) { return i == 0 ? 1.0 / 3.0 : 1.0 / 6.0; }
};

// Stencil of the isotropic wall-normal estimate: D3Q19 in 3D, D2Q9 in 2D.
template <int DIM> struct NormalStencil;
template <> struct NormalStencil<3> { using L = D3Q19; };
template <> struct NormalStencil<2> { using L = D2Q9; };

}  // namespace lbrbc
