// pkr_lattices.h -- compile-time discrete velocity sets of the high-order
// kinetic relaxation scheme.
//
// The velocity sets are those of the paper's Appendix ("Quadrature of the
// Boltzmann Equation"): the 1D sets of the N = 3, 5, 7 quadratures, the 3D set
// of Table "vector2" (111 vectors in 10 shells), their 2D tensor products,
// and the standard D3Q19 set of first-order lattice Boltzmann.  Velocities are
// generated here by constexpr code so that the sweep kernels see every
// component as an immediate after unrolling; they are ordered by symmetry
// class (the sorted absolute components), and every velocity of a class
// shares its quadrature weight and hence its phi_i and chi_i.
#pragma once
#include <cstdint>

namespace pkr {

#if defined(__CUDACC__)
#define PKR_HD __host__ __device__
#else
#define PKR_HD
#endif

struct V3 {
    int x, y, z;
};

template <int Q_>
struct VelTable {
    V3 v[Q_];
    int cls[Q_];   // symmetry class of each velocity (0 .. ncls-1)
    int key[Q_];   // sorted |components| packed as hi*256 + mid*16 + lo
    int ncls;
    int reach;
};

constexpr int cabs(int a) { return a < 0 ? -a : a; }

constexpr int class_key(V3 v)
{
    int a = cabs(v.x), b = cabs(v.y), c = cabs(v.z);
    // sort descending
    if (a < b) { int t = a; a = b; b = t; }
    if (b < c) { int t = b; b = c; c = t; }
    if (a < b) { int t = a; a = b; b = t; }
    return a * 256 + b * 16 + c;
}

template <int Q>
constexpr void finish_table(VelTable<Q>& t)
{
    // stable insertion sort by class key, then number the classes
    for (int i = 0; i < Q; ++i) t.key[i] = class_key(t.v[i]);
    for (int i = 1; i < Q; ++i) {
        V3 v = t.v[i];
        int k = t.key[i];
        int j = i - 1;
        while (j >= 0 && t.key[j] > k) {
            t.v[j + 1] = t.v[j];
            t.key[j + 1] = t.key[j];
            --j;
        }
        t.v[j + 1] = v;
        t.key[j + 1] = k;
    }
    int c = -1, prev = -1, r = 0;
    for (int i = 0; i < Q; ++i) {
        if (t.key[i] != prev) { ++c; prev = t.key[i]; }
        t.cls[i] = c;
        int m = cabs(t.v[i].x);
        if (cabs(t.v[i].y) > m) m = cabs(t.v[i].y);
        if (cabs(t.v[i].z) > m) m = cabs(t.v[i].z);
        if (m > r) r = m;
    }
    t.ncls = c + 1;
    t.reach = r;
}

// All distinct sign/permutation images of the representatives, in order.
template <int Q>
constexpr VelTable<Q> from_shells(const int (*reps)[3], int nreps)
{
    VelTable<Q> t{};
    int n = 0;
    const int perm[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
    for (int r = 0; r < nreps; ++r)
        for (int p = 0; p < 6; ++p)
            for (int s = 0; s < 8; ++s) {
                int c[3] = {reps[r][perm[p][0]], reps[r][perm[p][1]], reps[r][perm[p][2]]};
                V3 v{(s & 1) ? -c[0] : c[0], (s & 2) ? -c[1] : c[1], (s & 4) ? -c[2] : c[2]};
                bool dup = false;
                for (int j = 0; j < n; ++j)
                    if (t.v[j].x == v.x && t.v[j].y == v.y && t.v[j].z == v.z) dup = true;
                if (!dup && n < Q) t.v[n++] = v;
            }
    finish_table(t);
    return t;
}

// 1D set {0, +-b_1, +-b_2, ...} as a table with velocities along x.
template <int Q>
constexpr VelTable<Q> line(const int* base)
{
    VelTable<Q> t{};
    t.v[0] = V3{0, 0, 0};
    for (int k = 0; k < (Q - 1) / 2; ++k) {
        t.v[1 + 2 * k] = V3{base[k], 0, 0};
        t.v[2 + 2 * k] = V3{-base[k], 0, 0};
    }
    finish_table(t);
    return t;
}

// Tensor product of a 1D set with itself in the (x, y) plane.
template <int Q, int Q1>
constexpr VelTable<Q> square(const int* base)
{
    int vs[Q1] = {};
    for (int k = 0; k < (Q1 - 1) / 2; ++k) {
        vs[1 + 2 * k] = base[k];
        vs[2 + 2 * k] = -base[k];
    }
    VelTable<Q> t{};
    int n = 0;
    for (int a = 0; a < Q1; ++a)
        for (int b = 0; b < Q1; ++b) t.v[n++] = V3{vs[a], vs[b], 0};
    finish_table(t);
    return t;
}

// Positive speeds of the paper's 1D sets (Appendix): N = 3 (and 1): {1, 3};
// N = 5: {1, 2, 3, 5}; N = 7: {1, ..., 6}.
constexpr int kBase5[2] = {1, 3};
constexpr int kBase9[4] = {1, 2, 3, 5};
constexpr int kBase13[6] = {1, 2, 3, 4, 5, 6};

// Shell representatives of Table "vector2" (D3Q111) and of D3Q19.
constexpr int kShells111[10][3] = {{0, 0, 0}, {1, 0, 0}, {1, 1, 0}, {3, 3, 3}, {3, 3, 0},
                                   {3, 1, 0}, {2, 2, 0}, {2, 1, 1}, {2, 0, 0}, {3, 0, 0}};
constexpr int kShells19[3][3] = {{0, 0, 0}, {1, 0, 0}, {1, 1, 0}};

struct D1Q5 {
    static constexpr int Q = 5, DIM = 1;
    static constexpr VelTable<Q> T = line<Q>(kBase5);
};
struct D1Q9 {
    static constexpr int Q = 9, DIM = 1;
    static constexpr VelTable<Q> T = line<Q>(kBase9);
};
struct D1Q13 {
    static constexpr int Q = 13, DIM = 1;
    static constexpr VelTable<Q> T = line<Q>(kBase13);
};
struct D2Q25 {
    static constexpr int Q = 25, DIM = 2;
    static constexpr VelTable<Q> T = square<Q, 5>(kBase5);
};
struct D2Q81 {
    static constexpr int Q = 81, DIM = 2;
    static constexpr VelTable<Q> T = square<Q, 9>(kBase9);
};
struct D2Q169 {
    static constexpr int Q = 169, DIM = 2;
    static constexpr VelTable<Q> T = square<Q, 13>(kBase13);
};
struct D3Q19 {
    static constexpr int Q = 19, DIM = 3;
    static constexpr VelTable<Q> T = from_shells<Q>(kShells19, 3);
};
struct D3Q111 {
    static constexpr int Q = 111, DIM = 3;
    static constexpr VelTable<Q> T = from_shells<Q>(kShells111, 10);
};

// Upper bound on the number of symmetry classes of any set above (D2Q169: 28).
constexpr int kMaxClasses = 32;

}  // namespace pkr
