// Point-to-face distance for the faces of the Freudenthal triangulation,
// in the normalised dose-distance space of Eq. (1) (Section 2.1).
//
// Every face of the triangulation is a vertex chain p + u0 < p + u1 < ... <
// p + um with u0 = 0 and the u's nested 0/1 masks over the axes.  A cell
// (lower corner p) owns the faces whose lowest vertex is p: 1 vertex, 7 edges,
// 12 triangles and 6 tetrahedra in 3D; 1 + 3 + 2 in 2D.  Every owned face
// lies inside the cell box [p, p + 1], which is what makes the radial early
// exit of Algorithm A1 (step 4b-ii) exact with a box-distance key.
//
// Projection (the normal equations of Section 2.1, solved in closed form).
// Take the reference point as the origin, q(u) = D_e(p+u)/dD - D_r/dD the
// relative dose of vertex u and s0 = (p - v) * h / dta the spatial position of
// the lowest vertex.  Use the chain increments e_i = w_i - w_{i-1} as the
// basis of the face.  Their spatial parts are the axis sets A_i = u_i \ u_{i-1},
// which are disjoint, so they are orthogonal with squared lengths
// sigma_i^2 = sum_{a in A_i} (h_a/dta)^2 = 1/kappa_i.  With d_i = q(u_i) -
// q(u_{i-1}) the Gram matrix is diag(sigma^2) + d d^T and the projection of
// the origin onto the face's affine hull has, in closed form,
//     D     = 1 + sum_i d_i^2 kappa_i
//     L     = q(0) + sum_i d_i beta_i,  beta_i = -(s0 . e_i^spatial) kappa_i
//     mu_i  = beta_i - (L / D) d_i kappa_i          (coefficient of e_i)
//     dist2 = rho^2 + L^2 / D
// where rho^2 is the squared spatial distance from the origin to the face's
// spatial affine subspace.  The point lies in the face iff
//     1 >= mu_1 >= mu_2 >= ... >= mu_m >= 0.
// beta and rho^2 depend only on the integer cell offset and the spacing and
// are formed without cancellation (Lagrange's identity for the 2- and 3-axis
// blocks), so the whole evaluation is well conditioned in FP32.
//
// Taking the minimum over every face with a valid projection gives the
// distance to the closed surface (the nearest point lies in the relative
// interior of exactly one face, where it is that face's projection).  This
// is the paper's GPU choice of evaluating all simplexes instead of Ju's
// recursion (Section 2.2).
#pragma once
#include <cstdint>
#include <tuple>
#include <utility>

namespace gk {

constexpr float kInf = __builtin_huge_valf();

__host__ __device__ __forceinline__ float fma_(float a, float b, float c) { return fmaf(a, b, c); }
__host__ __device__ __forceinline__ double fma_(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float div_(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double div_(double a, double b) { return a / b; }
__device__ __forceinline__ float min_(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ double min_(double a, double b) { return fmin(a, b); }

// Per-cell spatial constants, indexed by axis-subset mask (bit 0 = x); 2D
// problems use the first four entries.
template <typename T>
struct CellGeom {
    T beta[8];   // beta_A = -(sum_{a in A} hn2_a c_a) kappa_A
    T br[8];     // rho^2 contribution of an increment spanning A
    T tsum[8];   // sum over axes NOT in the mask of (hn_a c_a)^2
};

// Uniform per-problem constants.
template <typename T>
struct MetricT {
    T hn2[3];      // (h_a / dta)^2 for a = x, y, z
    T kappa[8];    // 1 / sum_{a in A} hn2_a for each axis subset A (index 0 unused)
};
using Metric = MetricT<float>;

// Cell constants for the lower-corner offset c (voxel units from the
// reference point; integer on a coincident grid, real otherwise).
template <int N, typename T, typename C>
__host__ __device__ __forceinline__ void cell_geom(C cx, C cy, C cz, const MetricT<T>& mt,
                                          CellGeom<T>& g)
{
    const T c[3] = {T(cx), T(cy), T(cz)};
    T t[3] = {T(0), T(0), T(0)};
#pragma unroll
    for (int a = 0; a < N; ++a) t[a] = mt.hn2[a] * c[a] * c[a];
#pragma unroll
    for (int A = 0; A < 8; ++A) { g.beta[A] = T(0); g.br[A] = T(0); g.tsum[A] = T(0); }
#pragma unroll
    for (int A = 1; A < (1 << N); ++A) {
        T s = T(0);
#pragma unroll
        for (int a = 0; a < N; ++a)
            if (A & (1 << a)) s = fma_(mt.hn2[a], c[a], s);
        g.beta[A] = -s * mt.kappa[A];
    }
#pragma unroll
    for (int M = 0; M < (1 << N); ++M) {
        T s = T(0);
#pragma unroll
        for (int a = 0; a < N; ++a)
            if (!(M & (1 << a))) s += t[a];
        g.tsum[M] = s;
    }
    // two-axis blocks: hn2_a hn2_b (c_a - c_b)^2 kappa_ab (Lagrange's identity)
#pragma unroll
    for (int a = 0; a < N; ++a)
#pragma unroll
        for (int b = a + 1; b < N; ++b) {
            const T dc = c[a] - c[b];
            g.br[(1 << a) | (1 << b)] = mt.hn2[a] * mt.hn2[b] * dc * dc * mt.kappa[(1 << a) | (1 << b)];
        }
    if constexpr (N == 3) {
        const T dxy = c[0] - c[1], dxz = c[0] - c[2], dyz = c[1] - c[2];
        T s = mt.hn2[0] * mt.hn2[1] * dxy * dxy;
        s = fma_(mt.hn2[0] * mt.hn2[2], dxz * dxz, s);
        s = fma_(mt.hn2[1] * mt.hn2[2], dyz * dyz, s);
        g.br[7] = s * mt.kappa[7];
    }
}

// Projection of the origin onto the owned face with chain (U1[, U2[, U3]]).
// d2 is the squared distance, or +inf when the projection falls outside the
// face or the face leaves the grid; mu are the coefficients of the chain
// increments (the foot point is s0 + sum_i mu_i e_i).
//
// Near-singular Gram matrices.  With the increments scaled to unit spatial
// length the Gram matrix is I + g g^T, whose normalised determinant
// det(G) / prod(G_ii) = D / prod_i (1 + g_i^2) with D = 1 + |g|^2.  Since
// every factor 1 + g_i^2 <= D, the ratio is >= D^(1 - M), so it can only fall
// below tau when D > tau^(-1/2) (M = 3) or tau^(-1) (M = 2).  The face
// therefore only raises `ill` when D > dmax = tau^(-1/2); the caller then
// applies the exact test (cell_gram_ill) before redoing the cell in FP64.
template <typename T>
struct FaceFoot {
    T d2, mu1, mu2, mu3;
};

template <int M, int U1, int U2, int U3, typename T>
__device__ __forceinline__ FaceFoot<T> face_core(const T (&q)[8], uint32_t ok, const CellGeom<T>& g,
                                                 const T (&kappa)[8], T dmax, bool& ill)
{
    constexpr int UM = M == 1 ? U1 : (M == 2 ? U2 : U3);
    constexpr int A1 = U1, A2 = U2 ^ U1, A3 = U3 ^ U2;
    const T d1 = q[U1] - q[0];
    const T k1 = d1 * kappa[A1];
    T D = fma_(d1, k1, T(1));
    T L = fma_(d1, g.beta[A1], q[0]);
    T rho2 = g.tsum[UM] + g.br[A1];
    T d2 = T(0), k2 = T(0), d3 = T(0), k3 = T(0);
    if constexpr (M >= 2) {
        d2 = q[U2] - q[U1];
        k2 = d2 * kappa[A2];
        D = fma_(d2, k2, D);
        L = fma_(d2, g.beta[A2], L);
        rho2 += g.br[A2];
    }
    if constexpr (M >= 3) {
        d3 = q[U3] - q[U2];
        k3 = d3 * kappa[A3];
        D = fma_(d3, k3, D);
        L = fma_(d3, g.beta[A3], L);
        rho2 += g.br[A3];
    }
    const T r = div_(L, D);
    FaceFoot<T> f;
    f.mu1 = fma_(-r, k1, g.beta[A1]);
    f.mu2 = T(0);
    f.mu3 = T(0);
    bool valid = f.mu1 <= T(1);
    T last = f.mu1;
    if constexpr (M >= 2) {
        f.mu2 = fma_(-r, k2, g.beta[A2]);
        valid = valid && (f.mu1 >= f.mu2);
        last = f.mu2;
        if constexpr (M >= 3) {
            f.mu3 = fma_(-r, k3, g.beta[A3]);
            valid = valid && (f.mu2 >= f.mu3);
            last = f.mu3;
        }
        ill = ill || (D > dmax);
    }
    valid = valid && (last >= T(0)) && ((ok >> UM) & 1u);
    f.d2 = valid ? fma_(L, r, rho2) : T(kInf);
    return f;
}

template <int M, int U1, int U2, int U3, typename T>
__device__ __forceinline__ T face_d2(const T (&q)[8], uint32_t ok, const CellGeom<T>& g,
                                     const T (&kappa)[8], T dmax, bool& ill)
{
    return face_core<M, U1, U2, U3, T>(q, ok, g, kappa, dmax, ill).d2;
}

template <int M, int U1, int U2, int U3>
struct Face {};

template <int N>
struct FaceList;

template <>
struct FaceList<2> {
    using type = std::tuple<Face<1, 1, 0, 0>, Face<1, 2, 0, 0>, Face<1, 3, 0, 0>,
                            Face<2, 1, 3, 0>, Face<2, 2, 3, 0>>;
};

template <>
struct FaceList<3> {
    // depth-first over the chain tree 0 -> u1 -> u2 -> u3, so that the
    // prefix terms of a chain are consumed by its extensions right away
    using type = std::tuple<
        Face<1, 1, 0, 0>, Face<2, 1, 3, 0>, Face<3, 1, 3, 7>, Face<2, 1, 5, 0>, Face<3, 1, 5, 7>,
        Face<2, 1, 7, 0>,
        Face<1, 2, 0, 0>, Face<2, 2, 3, 0>, Face<3, 2, 3, 7>, Face<2, 2, 6, 0>, Face<3, 2, 6, 7>,
        Face<2, 2, 7, 0>,
        Face<1, 4, 0, 0>, Face<2, 4, 5, 0>, Face<3, 4, 5, 7>, Face<2, 4, 6, 0>, Face<3, 4, 6, 7>,
        Face<2, 4, 7, 0>,
        Face<1, 3, 0, 0>, Face<2, 3, 7, 0>, Face<1, 5, 0, 0>, Face<2, 5, 7, 0>,
        Face<1, 6, 0, 0>, Face<2, 6, 7, 0>, Face<1, 7, 0, 0>>;
};

// Number of owned faces per cell (including the vertex).
template <int N>
constexpr int kFacesPerCell = N == 3 ? 26 : 6;

template <typename T, int M, int U1, int U2, int U3>
__device__ __forceinline__ void apply_face(Face<M, U1, U2, U3>, const T (&q)[8], uint32_t ok,
                                           const CellGeom<T>& g, const T (&kappa)[8], T dmax,
                                           T& best, bool& ill)
{
    best = min_(best, face_d2<M, U1, U2, U3, T>(q, ok, g, kappa, dmax, ill));
}

template <typename T, typename... Fs>
__device__ __forceinline__ void apply_all(std::tuple<Fs...>*, const T (&q)[8], uint32_t ok,
                                          const CellGeom<T>& g, const T (&kappa)[8], T dmax,
                                          T& best, bool& ill)
{
    (apply_face(Fs{}, q, ok, g, kappa, dmax, best, ill), ...);
}

// Minimum squared distance over all faces owned by one cell.  q holds the
// relative normalised doses of the cell's 2^N vertices (index = axis mask;
// entries of vertices outside the grid must be finite), ok has bit u set when
// vertex u lies inside the grid (bit 0 must be set).
template <int N, typename T>
__device__ __forceinline__ T cell_min_d2(const T (&q)[8], uint32_t ok, const CellGeom<T>& g,
                                         const MetricT<T>& mt, T dmax, T best, bool& ill)
{
    best = min_(best, fma_(q[0], q[0], g.tsum[0]));            // the vertex itself
    apply_all<T>((typename FaceList<N>::type*)nullptr, q, ok, g, mt.kappa, dmax, best, ill);
    return best;
}

// Exact near-singularity test of the cell's faces: det(G)/prod(G_ii) < tau.
template <int M, int U1, int U2, int U3>
__device__ __forceinline__ bool gram_ill_face(Face<M, U1, U2, U3>, const float (&q)[8], uint32_t ok,
                                              const float (&kappa)[8], float tau)
{
    if constexpr (M < 2) {
        return false;
    } else {
        constexpr int UM = M == 2 ? U2 : U3;
        constexpr int A1 = U1, A2 = U2 ^ U1, A3 = U3 ^ U2;
        if (!((ok >> UM) & 1u)) return false;
        const float d1 = q[U1] - q[0], d2 = q[U2] - q[U1];
        const float e1 = fmaf(d1 * kappa[A1], d1, 1.f), e2 = fmaf(d2 * kappa[A2], d2, 1.f);
        float D = e1 + e2 - 1.f, prod = e1 * e2;
        if constexpr (M >= 3) {
            const float d3 = q[U3] - q[U2];
            const float e3 = fmaf(d3 * kappa[A3], d3, 1.f);
            D += e3 - 1.f;
            prod *= e3;
        }
        return D < tau * prod;
    }
}

template <typename... Fs>
__device__ __forceinline__ bool gram_ill_all(std::tuple<Fs...>*, const float (&q)[8], uint32_t ok,
                                             const float (&kappa)[8], float tau)
{
    return (gram_ill_face(Fs{}, q, ok, kappa, tau) || ...);
}

template <int N>
__device__ __forceinline__ bool cell_gram_ill(const float (&q)[8], uint32_t ok, const float (&kappa)[8],
                                           float tau)
{
    return gram_ill_all((typename FaceList<N>::type*)nullptr, q, ok, kappa, tau);
}

// Argmin variant: the minimum over the cell's faces of the squared distance
// and the foot point, in voxel units relative to the cell's lower corner.
template <typename T, int M, int U1, int U2, int U3>
__device__ __forceinline__ void arg_face(Face<M, U1, U2, U3>, const T (&q)[8], uint32_t ok,
                                         const CellGeom<T>& g, const T (&kappa)[8], T& best,
                                         T (&foot)[3])
{
    bool ill = false;
    const FaceFoot<T> f = face_core<M, U1, U2, U3, T>(q, ok, g, kappa, T(kInf), ill);
    if (f.d2 < best) {
        best = f.d2;
        constexpr int A1 = U1, A2 = U2 ^ U1, A3 = U3 ^ U2;
#pragma unroll
        for (int a = 0; a < 3; ++a)
            foot[a] = ((A1 >> a) & 1 ? f.mu1 : T(0)) + (M >= 2 && ((A2 >> a) & 1) ? f.mu2 : T(0)) +
                      (M >= 3 && ((A3 >> a) & 1) ? f.mu3 : T(0));
    }
}

template <typename T, typename... Fs>
__device__ __forceinline__ void arg_all(std::tuple<Fs...>*, const T (&q)[8], uint32_t ok,
                                        const CellGeom<T>& g, const T (&kappa)[8], T& best,
                                        T (&foot)[3])
{
    (arg_face(Fs{}, q, ok, g, kappa, best, foot), ...);
}

template <int N, typename T>
__device__ __forceinline__ void cell_argmin(const T (&q)[8], uint32_t ok, const CellGeom<T>& g,
                                            const MetricT<T>& mt, T& best, T (&foot)[3])
{
    const T dv = fma_(q[0], q[0], g.tsum[0]);
    if (dv < best) {
        best = dv;
        foot[0] = foot[1] = foot[2] = T(0);
    }
    arg_all<T>((typename FaceList<N>::type*)nullptr, q, ok, g, mt.kappa, best, foot);
}

}  // namespace gk
