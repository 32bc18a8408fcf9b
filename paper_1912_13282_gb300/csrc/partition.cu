// Range partition of a node set for several GPUs (host code).  Stencil
// weights are independent per node (Section 2.2: one local system per node),
// so a node set splits into contiguous ranges of a space-filling order, one
// per GPU; each GPU also holds the halo -- the nodes of other ranges within a
// radius of its own -- so its stencils and its rows of an operator can be
// formed locally, and an explicit time step (Section 2.3.1) needs only the
// halo's values from the other GPUs.
//
//   mm_partition_morton  Morton (Z-order) permutation of the nodes and
//                        nparts balanced contiguous ranges of it.
//   mm_partition_halo    the nodes outside one range within `radius` of one
//                        of its nodes (grid binning, exact distances).
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <unordered_map>
#include <vector>

#include "mm.h"

namespace {

// Spreads the low `bits` bits of v so that consecutive bits are `stride`
// apart (bit b goes to position stride * b).
uint64_t spread_bits(uint64_t v, int bits, int stride) {
    uint64_t out = 0;
    for (int b = 0; b < bits; ++b) out |= ((v >> b) & 1ull) << (stride * b);
    return out;
}

bool bad_points(int dim, int64_t N, const double *pts) {
    if ((dim != 2 && dim != 3) || N < 1 || !pts) return true;
    for (int64_t i = 0; i < N * dim; ++i)
        if (!std::isfinite(pts[i])) return true;
    return false;
}

}  // namespace

extern "C" int mm_partition_morton(int dim, int64_t N, const double *h_pts, int nparts, int64_t *h_perm,
                                   int64_t *h_starts) {
    if (bad_points(dim, N, h_pts) || nparts < 1 || nparts > N || !h_perm || !h_starts) return MM_EBADARG;
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = 0; i < N; ++i)
        for (int a = 0; a < dim; ++a) {
            lo[a] = std::min(lo[a], h_pts[i * dim + a]);
            hi[a] = std::max(hi[a], h_pts[i * dim + a]);
        }
    // one common cell size for all axes (cubic cells keep ranges compact)
    double ext = 0.0;
    for (int a = 0; a < dim; ++a) ext = std::max(ext, hi[a] - lo[a]);
    const int bits = dim == 2 ? 31 : 21;
    const double cells = (double)((1ull << bits) - 1);
    const double scale = ext > 0.0 ? cells / ext : 0.0;
    std::vector<std::pair<uint64_t, int64_t>> key((size_t)N);
    for (int64_t i = 0; i < N; ++i) {
        uint64_t code = 0;
        for (int a = 0; a < dim; ++a) {
            double q = std::floor((h_pts[i * dim + a] - lo[a]) * scale);
            q = std::min(std::max(q, 0.0), cells);
            code |= spread_bits((uint64_t)q, bits, dim) << a;
        }
        key[(size_t)i] = {code, i};
    }
    std::sort(key.begin(), key.end());   // ties of the code by node index
    for (int64_t i = 0; i < N; ++i) h_perm[i] = key[(size_t)i].second;
    for (int p = 0; p <= nparts; ++p) h_starts[p] = (N * p) / nparts;
    return MM_OK;
}

extern "C" int mm_partition_halo(int dim, int64_t N, const double *h_pts, const int64_t *h_perm, int64_t begin,
                                 int64_t end, double radius, int64_t *h_halo, int64_t capacity,
                                 int64_t *nhalo) {
    if (bad_points(dim, N, h_pts) || !h_perm || !nhalo || begin < 0 || end < begin || end > N ||
        !(radius > 0.0) || !std::isfinite(radius) || capacity < 0 || (capacity > 0 && !h_halo))
        return MM_EBADARG;
    std::vector<char> in_range((size_t)N, 0);
    for (int64_t k = begin; k < end; ++k) {
        const int64_t i = h_perm[k];
        if (i < 0 || i >= N || in_range[(size_t)i]) return MM_EBADARG;   // not a permutation
        in_range[(size_t)i] = 1;
    }
    // the range's nodes binned on a grid of cell size `radius`: a node
    // within `radius` of a range node lies in one of the 3^dim cells around it
    auto cell_of = [&](const double *x, int64_t c[3]) {
        for (int a = 0; a < 3; ++a) c[a] = a < dim ? (int64_t)std::floor(x[a] / radius) : 0;
    };
    auto hash = [](int64_t a, int64_t b, int64_t c) {
        return (uint64_t)(a * 73856093LL) ^ (uint64_t)(b * 19349663LL) ^ (uint64_t)(c * 83492791LL);
    };
    std::unordered_map<uint64_t, std::vector<int64_t>> grid;
    for (int64_t k = begin; k < end; ++k) {
        const int64_t i = h_perm[k];
        int64_t c[3];
        cell_of(h_pts + i * dim, c);
        grid[hash(c[0], c[1], c[2])].push_back(i);
    }
    const double r2 = radius * radius;
    int64_t count = 0;
    for (int64_t j = 0; j < N; ++j) {
        if (in_range[(size_t)j]) continue;
        const double *xj = h_pts + j * dim;
        int64_t c[3];
        cell_of(xj, c);
        bool near = false;
        for (int64_t dx = -1; dx <= 1 && !near; ++dx)
            for (int64_t dy = -1; dy <= 1 && !near; ++dy)
                for (int64_t dz = (dim == 3 ? -1 : 0); dz <= (dim == 3 ? 1 : 0) && !near; ++dz) {
                    auto it = grid.find(hash(c[0] + dx, c[1] + dy, c[2] + dz));
                    if (it == grid.end()) continue;
                    for (int64_t i : it->second) {
                        double d2 = 0.0;
                        for (int a = 0; a < dim; ++a) {
                            const double t = xj[a] - h_pts[i * dim + a];
                            d2 += t * t;
                        }
                        if (d2 <= r2) { near = true; break; }
                    }
                }
        if (near) {
            if (count < capacity) h_halo[count] = j;
            ++count;
        }
    }
    *nhalo = count;
    return count <= capacity ? MM_OK : MM_EUNSUPPORTED;
}
