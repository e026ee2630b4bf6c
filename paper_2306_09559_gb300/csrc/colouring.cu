// Distance colourings of the periodic lattice for probing (host code only).
//
// Probing (paper Sec. 3.1 on the choice of p_3, Sec. 5 step 3d) finds Tr p(A)
// exactly from one probe vector per colour and spin-colour component when no
// two sites of one colour are coupled by p(A).  A polynomial of degree d in
// the nearest-neighbour Wilson matrix couples sites at most d hops apart, so
// the colouring must give different colours to any two sites whose hop
// distance on the periodic lattice is at most d: a distance-d colouring of
// the graph of A.
//
// Construction: greedy colouring (each site takes the smallest colour not
// used within distance d), with the sites visited in the order of a linear
// colouring key(x) = (a . x) mod q that is a valid distance-d colouring of
// the infinite lattice Z^4 (a . v != 0 mod q for every offset v with
// 1 <= |v|_1 <= d).  Where the extents are not multiples of q that key is
// not a colouring of the torus, but visiting its classes one after another
// packs the greedy colours close to q: about 110 colours for d = 4 on
// 24^3 x 32 and 8^4, against at least 41 (the 41 sites within distance 2 of
// one site are pairwise at most 4 hops apart) and 4096 colours of the
// period-8 colouring.  Deterministic: the key search uses a fixed integer
// sequence.
#include "mpmc.h"

#include <algorithm>
#include <cstdint>
#include <cstdlib>
#include <vector>

namespace {

struct Off {
    int d[4];
};

// Every offset v != 0 of Z^4 with |v|_1 <= dist.
std::vector<Off> ball(int dist) {
    std::vector<Off> out;
    for (int a = -dist; a <= dist; ++a)
        for (int b = -dist + std::abs(a); b <= dist - std::abs(a); ++b)
            for (int c = -dist + std::abs(a) + std::abs(b); c <= dist - std::abs(a) - std::abs(b); ++c) {
                const int r = dist - std::abs(a) - std::abs(b) - std::abs(c);
                for (int e = -r; e <= r; ++e)
                    if (a || b || c || e) out.push_back(Off{{a, b, c, e}});
            }
    return out;
}

// A linear key a . x mod q valid as a distance-dist colouring of Z^4, or q = 0 if none
// was found within the search budget.  q starts at the size of the ball of radius
// dist / 2, whose sites are pairwise within distance dist.
void linear_key(const std::vector<Off>& offs, int dist, int a[4], int* q_out) {
    *q_out = 0;
    const long long nb = std::max<long long>(2, (long long)ball(dist / 2).size() + 1);
    uint64_t state = 0x9E3779B97F4A7C15ull;
    long long budget = 60000000;                       // offset checks
    for (long long q = nb; q <= 4 * nb && budget > 0; ++q) {
        for (int trial = 0; trial < 4000 && budget > 0; ++trial) {
            int cand[4] = {1, 0, 0, 0};
            for (int i = 1; i < 4; ++i) {
                state = state * 6364136223846793005ull + 1442695040888963407ull;
                cand[i] = 1 + (int)((state >> 33) % (uint64_t)(q - 1));
            }
            bool ok = true;
            for (const Off& v : offs) {
                --budget;
                long long s = 0;
                for (int i = 0; i < 4; ++i) s += (long long)cand[i] * v.d[i];
                if (((s % q) + q) % q == 0) {
                    ok = false;
                    break;
                }
            }
            if (ok) {
                for (int i = 0; i < 4; ++i) a[i] = cand[i];
                *q_out = (int)q;
                return;
            }
        }
    }
}

}  // namespace

extern "C" int mpmc_colouring(const int dims[4], int distance, int* colours, int* ncolours) {
    if (!dims || !colours || !ncolours || distance < 0) return MPMC_EINVAL;
    long long V = 1;
    for (int i = 0; i < 4; ++i) {
        if (dims[i] < 2) return MPMC_EINVAL;
        V *= dims[i];
    }
    if (V > (1LL << 30)) return MPMC_EINVAL;
    const int lx = dims[0], ly = dims[1], lz = dims[2], lt = dims[3];
    if (distance == 0) {   // only a site with itself: one colour
        std::fill(colours, colours + V, 0);
        *ncolours = 1;
        return MPMC_OK;
    }
    // past half of every extent each site is within reach of every other: one colour per site
    if (distance >= lx / 2 + ly / 2 + lz / 2 + lt / 2) {
        for (long long s = 0; s < V; ++s) colours[s] = (int)s;
        *ncolours = (int)V;
        return MPMC_OK;
    }
    const std::vector<Off> offs = ball(distance);
    if ((double)V * (double)offs.size() > 8e9) return MPMC_ENOTSUP;   // too long a greedy pass
    // visiting order: by linear key, then by site index
    int a[4] = {0, 0, 0, 0}, q = 0;
    linear_key(offs, distance, a, &q);
    std::vector<int> order((size_t)V);
    for (long long s = 0; s < V; ++s) order[(size_t)s] = (int)s;
    if (q > 0) {
        std::vector<int> key((size_t)V);
        for (long long s = 0; s < V; ++s) {
            const long long x = s % lx, y = (s / lx) % ly, z = (s / ((long long)lx * ly)) % lz,
                            t = s / ((long long)lx * ly * lz);
            key[(size_t)s] = (int)((a[0] * x + a[1] * y + a[2] * z + a[3] * t) % q);
        }
        std::stable_sort(order.begin(), order.end(), [&](int u, int v) { return key[u] < key[v]; });
    }
    // greedy colouring; stamp[c] == s marks colour c as used near site s
    std::vector<int> col((size_t)V, -1);
    std::vector<long long> stamp;
    int maxc = 0;
    for (int s : order) {
        const int x = s % lx, y = (s / lx) % ly, z = (s / (lx * ly)) % lz, t = s / (lx * ly * lz);
        for (const Off& v : offs) {
            const int nx = ((x + v.d[0]) % lx + lx) % lx, ny = ((y + v.d[1]) % ly + ly) % ly;
            const int nz = ((z + v.d[2]) % lz + lz) % lz, nt = ((t + v.d[3]) % lt + lt) % lt;
            const int r = ((nt * lz + nz) * ly + ny) * lx + nx;
            if (r == s || col[(size_t)r] < 0) continue;
            const int c = col[(size_t)r];
            if ((size_t)c >= stamp.size()) stamp.resize((size_t)c + 1, -1);
            stamp[(size_t)c] = s;
        }
        int c = 0;
        while ((size_t)c < stamp.size() && stamp[(size_t)c] == s) ++c;
        col[(size_t)s] = c;
        maxc = std::max(maxc, c + 1);
    }
    std::copy(col.begin(), col.end(), colours);
    *ncolours = maxc;
    return MPMC_OK;
}
