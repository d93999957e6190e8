// Faces of the triangulation that contain the reference voxel's own node:
// the reduced closed form of the Section 2.1 projection used for the key-0
// cells (the 2^n cells whose box contains the voxel).
//
// Such a face is a chain through the voxel v,
//     v - W_b < ... < v - W_1 < v < v + V_1 < ... < v + V_a,
// with W_1 < ... < W_b and V_1 < ... < V_a strictly nested non-empty axis
// sets and W_b, V_a disjoint (a + b = m increments, 75 faces in 3D including
// the vertex itself, 13 in 2D).  In the general closed form (gamma_face.cuh)
// the chain starts at s0 = -W_b * h / dta, so beta_i = 1 for the b increments
// below v and 0 above it, rho^2 = 0, and L telescopes to the voxel's own
// relative dose q_v.  Multiplying D and the validity conditions by dD^2 (both
// sides of every condition scale alike) leaves, with g = D_e(v) - D_r and,
// per increment (edge) e with dose step Delta_e and axis set A_e,
//     t_e  = Delta_e^2 kappa_{A_e},      nu_e = g Delta_e kappa_{A_e},
//     D~   = dD^2 + sum_{e in face} t_e,
//     dist^2 = g^2 / D~,
// and the projection lies in the face iff, with M_i = beta_i D~ - nu_i and
// M_0 = D~, M_{m+1} = 0, the sequence M is non-increasing:
//     first edge below v: nu_1 >= 0          above v: nu_1 >= -D~
//     between edges:      nu_i <= nu_{i+1}   (+ D~ where the chain passes v)
//     last edge below v:  nu_m <= D~         above v: nu_m <= 0.
// The minimum over the faces through v is therefore g^2 / max D~ over the
// faces whose projection is valid (the vertex alone gives D~ = dD^2).  Every
// term is a product or a sum of non-negative terms: there is no cancellation,
// so FP32 needs no double-precision redo here.  Doses of nodes outside the
// grid are NaN, which makes every condition of a face that uses them false.
//
// The per-edge values are shared by all faces through the edge, so a 3D voxel
// costs 38 edges and 74 faces instead of 75 general face projections.
#pragma once
#include <cstdint>
#include <utility>

namespace gk {

// Node indices: 0 = v, U (1 .. 2^N - 1) = v - U, 2^N - 1 + U = v + U.
template <int N>
struct NearTable {
    static constexpr int NU = 1 << N;
    static constexpr int NPT = 2 * NU - 1;
    static constexpr int NE = N == 3 ? 38 : 10;
    static constexpr int NF = N == 3 ? 74 : 12;
    int ep[NE], eq[NE], ea[NE];   // edge: lower node, upper node, axis set
    int fm[NF], fb[NF];           // increments, increments below v
    int fe[NF][3];                // edges of the face, lowest first
    int ne, nf;                   // entries filled by the builder
};

template <int N>
constexpr int near_edge_index(const NearTable<N>& t, int p, int q)
{
    for (int e = 0; e < NearTable<N>::NE; ++e)
        if (t.ep[e] == p && t.eq[e] == q) return e;
    return -1;
}

template <int N>
constexpr NearTable<N> make_near_table()
{
    constexpr int NU = 1 << N;
    NearTable<N> t{};
    int ne = 0;
    for (int U = 1; U < NU; ++U)              // below v: v - U up to v - W, W a proper subset of U
        for (int W = 0; W < U; ++W)
            if ((W & U) == W) {
                t.ep[ne] = U;
                t.eq[ne] = W;
                t.ea[ne] = U ^ W;
                ++ne;
            }
    for (int V = 0; V < NU; ++V)              // above v: v + V up to v + W, W a proper superset
        for (int W = V + 1; W < NU; ++W)
            if ((V & W) == V) {
                t.ep[ne] = V ? NU - 1 + V : 0;
                t.eq[ne] = NU - 1 + W;
                t.ea[ne] = W ^ V;
                ++ne;
            }
    // strictly nested chains of non-empty axis sets (including the empty chain)
    int nch = 1, clen[32] = {0}, cs[32][3] = {};
    for (int i = 0; i < nch; ++i) {
        if (clen[i] == N) continue;
        const int last = clen[i] ? cs[i][clen[i] - 1] : 0;
        for (int s = 1; s < NU; ++s)
            if ((s & last) == last && s != last) {
                for (int j = 0; j < clen[i]; ++j) cs[nch][j] = cs[i][j];
                cs[nch][clen[i]] = s;
                clen[nch] = clen[i] + 1;
                ++nch;
            }
    }
    int nf = 0;
    for (int w = 0; w < nch; ++w)
        for (int v = 0; v < nch; ++v) {
            const int b = clen[w], a = clen[v];
            if (a + b == 0) continue;
            if (a && b && (cs[w][b - 1] & cs[v][a - 1])) continue;
            int node[7] = {}, k = 0;
            for (int j = b - 1; j >= 0; --j) node[k++] = cs[w][j];
            node[k++] = 0;
            for (int j = 0; j < a; ++j) node[k++] = NU - 1 + cs[v][j];
            t.fm[nf] = a + b;
            t.fb[nf] = b;
            for (int j = 0; j < 3; ++j) t.fe[nf][j] = j < a + b ? near_edge_index(t, node[j], node[j + 1]) : 0;
            ++nf;
        }
    t.ne = ne;
    t.nf = nf;
    return t;
}

template <int N>
inline constexpr NearTable<N> kNear = make_near_table<N>();

template <int N>
constexpr int near_below_edges()
{
    return N == 3 ? 19 : 5;
}

template <int N>
constexpr bool near_table_ok()
{
    constexpr NearTable<N> t = kNear<N>;
    if (t.ne != NearTable<N>::NE || t.nf != NearTable<N>::NF) return false;
    for (int e = 0; e < NearTable<N>::NE; ++e)
        if ((e < near_below_edges<N>()) != (t.ep[e] != 0 && t.ep[e] < (1 << N))) return false;
    for (int f = 0; f < NearTable<N>::NF; ++f)
        for (int j = 0; j < t.fm[f]; ++j)
            if (t.fe[f][j] < 0) return false;
    return true;
}
static_assert(near_table_ok<2>() && near_table_ok<3>(), "near-face table");

// Edges are numbered below-v first; faces are processed in three groups
// (below v only, above v only, through v) so that the below edges not used by
// the last group are dead before the above edges are formed.
template <int N, int E, bool BELOW>
__device__ __forceinline__ void near_edge(const float (&e)[2 * (1 << N) - 1], float g,
                                          const float (&kappa)[8], float (&t)[NearTable<N>::NE],
                                          float (&nu)[NearTable<N>::NE])
{
    if constexpr ((E < near_below_edges<N>()) == BELOW) {
        constexpr int p = kNear<N>.ep[E], q = kNear<N>.eq[E], a = kNear<N>.ea[E];
        const float dl = e[q] - e[p];
        const float k = dl * kappa[a];
        t[E] = dl * k;
        nu[E] = g * k;
    }
}

// group 0: below v only, 1: above v only, 2: through v from below to above
template <int N, int F, int GROUP>
__device__ __forceinline__ void near_face(const float (&t)[NearTable<N>::NE],
                                          const float (&nu)[NearTable<N>::NE], float D0, float& Dmax)
{
    constexpr int m = kNear<N>.fm[F], b = kNear<N>.fb[F];
    constexpr int group = b == m ? 0 : (b == 0 ? 1 : 2);
    if constexpr (group == GROUP) {
        constexpr int e0 = kNear<N>.fe[F][0], e1 = kNear<N>.fe[F][1], e2 = kNear<N>.fe[F][2];
        constexpr int el = m == 1 ? e0 : (m == 2 ? e1 : e2);
        float D = D0 + t[e0];
        if constexpr (m >= 2) D += t[e1];
        if constexpr (m >= 3) D += t[e2];
        bool ok = b >= 1 ? (nu[e0] >= 0.f) : (nu[e0] >= -D);
        if constexpr (m >= 2) ok = ok && (b == 1 ? nu[e0] <= nu[e1] + D : nu[e0] <= nu[e1]);
        if constexpr (m >= 3) ok = ok && (b == 2 ? nu[e1] <= nu[e2] + D : nu[e1] <= nu[e2]);
        ok = ok && (b == m ? nu[el] <= D : nu[el] <= 0.f);
        Dmax = ok ? fmaxf(Dmax, D) : Dmax;
    }
}

template <int N, int... Es, int... Fs>
__device__ __forceinline__ float near_faces(std::integer_sequence<int, Es...>,
                                            std::integer_sequence<int, Fs...>,
                                            const float (&e)[2 * (1 << N) - 1], float g,
                                            float dD, const float (&kappa)[8])
{
    float t[NearTable<N>::NE], nu[NearTable<N>::NE];
    const float D0 = dD * dD;
    // four running maxima (face F feeds Dm[F % 4]): the maximum does not
    // depend on the order, and four short chains replace one long one
    float Dm[4] = {D0, D0, D0, D0};
    (near_edge<N, Es, true>(e, g, kappa, t, nu), ...);
    (near_face<N, Fs, 0>(t, nu, D0, Dm[Fs & 3]), ...);
    (near_edge<N, Es, false>(e, g, kappa, t, nu), ...);
    (near_face<N, Fs, 1>(t, nu, D0, Dm[Fs & 3]), ...);
    (near_face<N, Fs, 2>(t, nu, D0, Dm[Fs & 3]), ...);
    return (g * g) / fmaxf(fmaxf(Dm[0], Dm[1]), fmaxf(Dm[2], Dm[3]));
}

// Squared gamma over the faces through voxel v (node tix of a staged tile
// with x stride 1 and row / plane strides SY / SZ).  inm / inp: bit a set when
// the neighbour at -1 / +1 along axis a is inside the grid.
template <int N, int SY, int SZ>
__device__ __forceinline__ float near_gamma2(const float* tile, int tix, uint32_t inm, uint32_t inp,
                                             float dr, float dD, const float (&kappa)[8])
{
    constexpr int NU = 1 << N;
    const float nan = __int_as_float(0x7fc00000);
    float e[2 * NU - 1];
    e[0] = tile[tix];
#pragma unroll
    for (int U = 1; U < NU; ++U) {
        const int off = (U & 1 ? 1 : 0) + (U & 2 ? SY : 0) + (U & 4 ? SZ : 0);
        e[U] = ((inm & U) == (uint32_t)U) ? tile[tix - off] : nan;
        e[NU - 1 + U] = ((inp & U) == (uint32_t)U) ? tile[tix + off] : nan;
    }
    return near_faces<N>(std::make_integer_sequence<int, NearTable<N>::NE>{},
                         std::make_integer_sequence<int, NearTable<N>::NF>{}, e, e[0] - dr, dD,
                         kappa);
}

}  // namespace gk
