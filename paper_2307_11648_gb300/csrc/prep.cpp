// Input preparation for libsic on the host: reverse-maximin ordering, later-ordered
// nearest-neighbour candidate lists, and supernode grouping.  Untimed set-up work
// (it produces the inputs of the device calls); exact and deterministic, so that the
// same points always give the same ordering, candidates and groups.
//
// Squared distances are summed coordinate by coordinate in FP64 and compiled
// without FMA contraction; ties are broken by index as stated in sic.h.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <thread>
#include <vector>

#include "sic.h"

namespace {

inline double dist2(const double* pts, int dim, int64_t a, int64_t b) {
    double s = 0.0;
    for (int c = 0; c < dim; ++c) {
        double d = pts[a * dim + c] - pts[b * dim + c];
        s += d * d;
    }
    return s;
}

int threads_of(int n_threads) {
    if (n_threads > 0) return n_threads;
    unsigned h = std::thread::hardware_concurrency();
    return h ? (int)h : 1;
}

template <typename F>
void parallel_for(int64_t count, int n_threads, int64_t chunk, F f) {
    int nt = threads_of(n_threads);
    if (nt <= 1 || count <= chunk) {
        for (int64_t i = 0; i < count; ++i) f(i);
        return;
    }
    std::atomic<int64_t> next(0);
    std::vector<std::thread> pool;
    for (int t = 0; t < nt; ++t)
        pool.emplace_back([&]() {
            for (;;) {
                int64_t b = next.fetch_add(chunk);
                if (b >= count) break;
                int64_t e = std::min(count, b + chunk);
                for (int64_t i = b; i < e; ++i) f(i);
            }
        });
    for (auto& th : pool) th.join();
}

// Uniform grid over a subset of points (given by their rows in pts).
struct Grid {
    int dim = 1;
    int g = 1;  // cells per dimension
    double lo[3] = {0, 0, 0}, h[3] = {1, 1, 1};
    std::vector<int64_t> start;  // cell offsets into items, size cells + 1
    std::vector<int64_t> items;  // rows, grouped by cell, ascending within a cell

    int64_t cells() const {
        int64_t c = 1;
        for (int d = 0; d < dim; ++d) c *= g;
        return c;
    }
    int cell_coord(double x, int d) const {
        double f = (x - lo[d]) / h[d];
        int c = (int)std::floor(f);
        return std::min(std::max(c, 0), g - 1);
    }
    int64_t flat(const int* c) const {
        int64_t f = 0;
        for (int d = dim - 1; d >= 0; --d) f = f * g + c[d];
        return f;
    }
    void build(const double* pts, int dim_, const int64_t* rows, int64_t count, double per_cell) {
        dim = dim_;
        double cellsf = std::max(1.0, (double)count / per_cell);
        g = std::max(1, (int)std::floor(std::pow(cellsf, 1.0 / dim) + 1e-9));
        if (g > 4096) g = 4096;
        for (int d = 0; d < dim; ++d) {
            double mn = INFINITY, mx = -INFINITY;
            for (int64_t i = 0; i < count; ++i) {
                double v = pts[rows[i] * dim + d];
                mn = std::min(mn, v);
                mx = std::max(mx, v);
            }
            if (count == 0) mn = 0, mx = 1;
            double span = mx - mn;
            if (!(span > 0)) span = 1.0;
            lo[d] = mn;
            h[d] = span / g * (1.0 + 1e-12);
        }
        int64_t nc = cells();
        start.assign(nc + 1, 0);
        std::vector<int64_t> cid(count);
        for (int64_t i = 0; i < count; ++i) {
            int c[3];
            for (int d = 0; d < dim; ++d) c[d] = cell_coord(pts[rows[i] * dim + d], d);
            cid[i] = flat(c);
            start[cid[i] + 1]++;
        }
        for (int64_t c = 0; c < nc; ++c) start[c + 1] += start[c];
        items.assign(count, 0);
        std::vector<int64_t> fill(start.begin(), start.end() - 1);
        for (int64_t i = 0; i < count; ++i) items[fill[cid[i]]++] = rows[i];
    }
};

// Indexed binary max-heap over points keyed by (d desc, index asc), with decrease-key.
struct MaxHeap {
    std::vector<int64_t> heap, where;
    const std::vector<double>* key;
    bool above(int64_t a, int64_t b) const {  // a should sit above b
        double ka = (*key)[a], kb = (*key)[b];
        return ka > kb || (ka == kb && a < b);
    }
    void swap_at(int64_t i, int64_t j) {
        std::swap(heap[i], heap[j]);
        where[heap[i]] = i;
        where[heap[j]] = j;
    }
    void sift_down(int64_t i) {
        int64_t n = (int64_t)heap.size();
        for (;;) {
            int64_t l = 2 * i + 1, r = l + 1, b = i;
            if (l < n && above(heap[l], heap[b])) b = l;
            if (r < n && above(heap[r], heap[b])) b = r;
            if (b == i) return;
            swap_at(i, b);
            i = b;
        }
    }
    int64_t pop() {
        int64_t top = heap[0];
        swap_at(0, (int64_t)heap.size() - 1);
        heap.pop_back();
        where[top] = -1;
        if (!heap.empty()) sift_down(0);
        return top;
    }
};

// ---- exact k nearest (min over targets) among positions >= first, by ring search ----

struct KeyPos {
    double key;
    int64_t pos;
    bool operator<(const KeyPos& o) const { return key < o.key || (key == o.key && pos < o.pos); }
};

// Suffix grids: level l holds positions [n - size_l, n), size_l = base * 2^l (capped at n).
struct SuffixGrids {
    std::vector<int64_t> size;
    std::vector<Grid> grid;
    void build(const double* pts, int64_t n, int dim, int64_t base, int n_threads) {
        for (int64_t s = std::min(base, n);; s = std::min(2 * s, n)) {
            size.push_back(s);
            if (s == n) break;
        }
        grid.resize(size.size());
        parallel_for((int64_t)size.size(), n_threads, 1, [&](int64_t l) {
            std::vector<int64_t> rows(size[l]);
            for (int64_t i = 0; i < size[l]; ++i) rows[i] = n - size[l] + i;
            grid[l].build(pts, dim, rows.data(), size[l], 2.0);
        });
    }
    const Grid& for_first(int64_t n, int64_t first) const {
        int64_t need = n - first;
        for (size_t l = 0; l < size.size(); ++l)
            if (size[l] >= need) return grid[l];
        return grid.back();
    }
};

int32_t knn_query(const double* pts, int64_t n, int dim, const SuffixGrids& sg, const int64_t* tg, int m,
                  int64_t first, int32_t C, int32_t* out, std::vector<KeyPos>& buf) {
    if (first >= n || C <= 0) return 0;
    const Grid& G = sg.for_first(n, first);
    int clo[3] = {0, 0, 0}, chi[3] = {0, 0, 0};
    for (int d = 0; d < dim; ++d) {
        double mn = INFINITY, mx = -INFINITY;
        for (int a = 0; a < m; ++a) {
            double v = pts[tg[a] * dim + d];
            mn = std::min(mn, v);
            mx = std::max(mx, v);
        }
        clo[d] = G.cell_coord(mn, d);
        chi[d] = G.cell_coord(mx, d);
    }
    double hmin = INFINITY;
    for (int d = 0; d < dim; ++d) hmin = std::min(hmin, G.h[d]);
    buf.clear();
    const int64_t avail = n - first;
    for (int ring = 0;; ++ring) {
        // visit cells at Chebyshev ring distance `ring` from the box [clo, chi]
        int lo[3], hi[3];
        bool covers_all = true;
        for (int d = 0; d < 3; ++d) {
            lo[d] = (d < dim) ? std::max(0, clo[d] - ring) : 0;
            hi[d] = (d < dim) ? std::min(G.g - 1, chi[d] + ring) : 0;
            if (d < dim && (clo[d] - ring > 0 || chi[d] + ring < G.g - 1)) covers_all = false;
        }
        int c[3];
        for (c[2] = lo[2]; c[2] <= hi[2]; ++c[2])
            for (c[1] = lo[1]; c[1] <= hi[1]; ++c[1])
                for (c[0] = lo[0]; c[0] <= hi[0]; ++c[0]) {
                    bool on_ring = false;
                    for (int d = 0; d < dim; ++d)
                        if (c[d] == clo[d] - ring || c[d] == chi[d] + ring) on_ring = true;
                    if (ring > 0 && !on_ring) continue;
                    int64_t f = G.flat(c);
                    for (int64_t p = G.start[f]; p < G.start[f + 1]; ++p) {
                        int64_t j = G.items[p];
                        if (j < first) continue;
                        double best = INFINITY;
                        for (int a = 0; a < m; ++a) {
                            double e = dist2(pts, dim, j, tg[a]);
                            if (e < best) best = e;
                        }
                        buf.push_back({best, j});
                    }
                }
        if (covers_all) break;
        if ((int64_t)buf.size() >= C) {
            double reach = ring * hmin;
            std::nth_element(buf.begin(), buf.begin() + (C - 1), buf.end());
            if (buf[C - 1].key <= reach * reach) break;
        }
        if ((int64_t)buf.size() >= avail) break;
    }
    int32_t take = (int32_t)std::min<int64_t>(C, (int64_t)buf.size());
    std::partial_sort(buf.begin(), buf.begin() + take, buf.end());
    for (int32_t t = 0; t < take; ++t) out[t] = (int32_t)buf[t].pos;
    return take;
}

}  // namespace

extern "C" sic_status sic_prep_maximin(const double* pts, int64_t n, int32_t dim, int64_t* order, double* ell2,
                                       int32_t n_threads) {
    (void)n_threads;
    if (!pts || !order || !ell2 || n < 1 || dim < 1 || dim > 3) return SIC_ERR_INVALID;
    for (int64_t i = 0; i < n * dim; ++i)
        if (!std::isfinite(pts[i])) return SIC_ERR_INVALID;
    std::vector<double> d(n);
    std::vector<char> placed(n, 0);
    placed[0] = 1;
    order[n - 1] = 0;
    ell2[n - 1] = INFINITY;
    if (n == 1) return SIC_OK;
    for (int64_t j = 0; j < n; ++j) d[j] = dist2(pts, dim, j, 0);
    std::vector<int64_t> all(n);
    for (int64_t i = 0; i < n; ++i) all[i] = i;
    Grid G;
    G.build(pts, dim, all.data(), n, 2.0);
    MaxHeap H;
    H.key = &d;
    H.where.assign(n, -1);
    H.heap.reserve(n);
    for (int64_t j = 1; j < n; ++j) {
        H.where[j] = (int64_t)H.heap.size();
        H.heap.push_back(j);
    }
    for (int64_t i = (int64_t)H.heap.size() / 2 - 1; i >= 0; --i) H.sift_down(i);
    for (int64_t pos = n - 2; pos >= 0; --pos) {
        int64_t sel = H.pop();
        order[pos] = sel;
        ell2[pos] = d[sel];
        placed[sel] = 1;
        double r = std::sqrt(d[sel]);
        int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
        for (int c = 0; c < dim; ++c) {
            double x = pts[sel * dim + c];
            lo[c] = std::max(0, G.cell_coord(x - r, c) - 1);
            hi[c] = std::min(G.g - 1, G.cell_coord(x + r, c) + 1);
        }
        int c[3];
        for (c[2] = lo[2]; c[2] <= hi[2]; ++c[2])
            for (c[1] = lo[1]; c[1] <= hi[1]; ++c[1])
                for (c[0] = lo[0]; c[0] <= hi[0]; ++c[0]) {
                    int64_t f = G.flat(c);
                    for (int64_t p = G.start[f]; p < G.start[f + 1]; ++p) {
                        int64_t j = G.items[p];
                        if (placed[j]) continue;
                        double e = dist2(pts, dim, j, sel);
                        if (e < d[j]) {
                            d[j] = e;
                            H.sift_down(H.where[j]);
                        }
                    }
                }
    }
    return SIC_OK;
}

extern "C" sic_status sic_prep_candidates_columns(const double* pts, int64_t n, int32_t dim, int32_t n_cand,
                                                  int64_t* cand_ptr, int32_t* cand_idx, int32_t n_threads) {
    if (!pts || !cand_ptr || !cand_idx || n < 1 || dim < 1 || dim > 3 || n_cand < 0) return SIC_ERR_INVALID;
    SuffixGrids sg;
    sg.build(pts, n, dim, std::max<int64_t>(256, 4LL * n_cand), n_threads);
    std::vector<int32_t> cnt(n, 0);
    parallel_for(n, n_threads, 256, [&](int64_t i) {
        thread_local std::vector<KeyPos> buf;
        int64_t t = i;
        cnt[i] = knn_query(pts, n, dim, sg, &t, 1, i + 1, n_cand, cand_idx + i * (int64_t)n_cand, buf);
    });
    // compact in place (each list moves to an offset <= its own)
    cand_ptr[0] = 0;
    for (int64_t i = 0; i < n; ++i) {
        int64_t src = i * (int64_t)n_cand, dst = cand_ptr[i];
        if (dst != src) std::copy(cand_idx + src, cand_idx + src + cnt[i], cand_idx + dst);
        cand_ptr[i + 1] = dst + cnt[i];
    }
    return SIC_OK;
}

extern "C" sic_status sic_prep_candidates_targets(const double* pts, int64_t n, int32_t dim, int64_t n_targets,
                                                  int32_t n_cand, int64_t* cand_ptr, int32_t* cand_idx,
                                                  int32_t n_threads) {
    if (!pts || !cand_ptr || !cand_idx || n < 1 || dim < 1 || dim > 3 || n_cand < 0 || n_targets < 0 ||
        n_targets > n)
        return SIC_ERR_INVALID;
    cand_ptr[0] = 0;
    if (n_targets == 0) return SIC_OK;
    SuffixGrids sg;
    sg.build(pts, n, dim, std::max<int64_t>(256, n - n_targets), n_threads);
    std::vector<int32_t> cnt(n_targets, 0);
    parallel_for(n_targets, n_threads, 256, [&](int64_t i) {
        thread_local std::vector<KeyPos> buf;
        int64_t t = i;
        cnt[i] = knn_query(pts, n, dim, sg, &t, 1, n_targets, n_cand, cand_idx + i * (int64_t)n_cand, buf);
    });
    for (int64_t i = 0; i < n_targets; ++i) {
        int64_t src = i * (int64_t)n_cand, dst = cand_ptr[i];
        if (dst != src) std::copy(cand_idx + src, cand_idx + src + cnt[i], cand_idx + dst);
        cand_ptr[i + 1] = dst + cnt[i];
    }
    return SIC_OK;
}

extern "C" sic_status sic_prep_groups(const double* pts, const double* ell2, int64_t n, int32_t dim, int32_t K,
                                      double lambda, int32_t mmin, int32_t mmax, int64_t* members,
                                      int64_t* grp_ptr, int64_t* n_grp, int32_t n_threads) {
    if (!pts || !ell2 || !members || !grp_ptr || !n_grp || n < 1 || dim < 1 || dim > 3 || K < 0 || mmax < 1 ||
        mmin < 0 || !(lambda >= 1.0))
        return SIC_ERR_INVALID;
    const double lambda2 = lambda * lambda;
    SuffixGrids sg;
    sg.build(pts, n, dim, std::max<int64_t>(256, 4LL * K), n_threads);
    std::vector<char> done(n, 0);
    std::vector<int32_t> nb(std::max(K, 1));
    std::vector<KeyPos> buf;
    std::vector<int64_t> first;
    first.push_back(0);
    int64_t w = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (done[i]) continue;
        int32_t gm = 0;
        members[w + gm++] = i;
        done[i] = 1;
        int64_t t = i;
        int32_t cnt = knn_query(pts, n, dim, sg, &t, 1, i + 1, K, nb.data(), buf);
        for (int32_t q = 0; q < cnt && gm < mmax; ++q) {
            int64_t j = nb[q];
            if (done[j]) continue;
            if (ell2[j] <= lambda2 * ell2[i]) {
                members[w + gm++] = j;
                done[j] = 1;
            }
        }
        w += gm;
        first.push_back(w);
    }
    int64_t ng = (int64_t)first.size() - 1, out = 0;
    grp_ptr[0] = 0;
    for (int64_t q = 0; q < ng; ++q) {
        int64_t sz = first[q + 1] - first[q];
        if (out > 0 && sz < mmin && first[q + 1] - grp_ptr[out - 1] <= mmax)
            grp_ptr[out] = first[q + 1];
        else
            grp_ptr[++out] = first[q + 1];
    }
    for (int64_t q = 0; q < out; ++q) std::sort(members + grp_ptr[q], members + grp_ptr[q + 1]);
    *n_grp = out;
    return SIC_OK;
}

extern "C" sic_status sic_prep_candidates_groups(const double* pts, int64_t n, int32_t dim, const int64_t* grp_ptr,
                                                 int64_t n_grp, int32_t n_cand, int64_t* cand_ptr,
                                                 int32_t* cand_idx, int32_t n_threads) {
    if (!pts || !grp_ptr || !cand_ptr || !cand_idx || n < 1 || dim < 1 || dim > 3 || n_grp < 1 || n_cand < 0)
        return SIC_ERR_INVALID;
    SuffixGrids sg;
    sg.build(pts, n, dim, std::max<int64_t>(256, 4LL * n_cand), n_threads);
    std::vector<int32_t> cnt(n_grp, 0);
    parallel_for(n_grp, n_threads, 16, [&](int64_t g) {
        thread_local std::vector<KeyPos> buf;
        thread_local std::vector<int64_t> tg;
        int64_t a = grp_ptr[g], b = grp_ptr[g + 1];
        tg.resize(b - a);
        for (int64_t i = a; i < b; ++i) tg[i - a] = i;
        cnt[g] = knn_query(pts, n, dim, sg, tg.data(), (int)(b - a), b, n_cand, cand_idx + g * (int64_t)n_cand, buf);
    });
    cand_ptr[0] = 0;
    for (int64_t g = 0; g < n_grp; ++g) {
        int64_t src = g * (int64_t)n_cand, dst = cand_ptr[g];
        if (dst != src) std::copy(cand_idx + src, cand_idx + src + cnt[g], cand_idx + dst);
        cand_ptr[g + 1] = dst + cnt[g];
    }
    return SIC_OK;
}

extern "C" sic_status sic_prep_candidates_partial(const double* pts, int64_t n, int32_t dim, const int64_t* members,
                                                  const int64_t* grp_ptr, int64_t n_grp, int32_t n_cand,
                                                  int64_t* cand_ptr, int32_t* cand_idx, int32_t n_threads) {
    if (!pts || !members || !grp_ptr || !cand_ptr || !cand_idx || n < 1 || dim < 1 || dim > 3 || n_grp < 1 ||
        n_cand < 0)
        return SIC_ERR_INVALID;
    for (int64_t g = 0; g < n_grp; ++g) {
        if (grp_ptr[g + 1] <= grp_ptr[g]) return SIC_ERR_INVALID;
        for (int64_t a = grp_ptr[g]; a < grp_ptr[g + 1]; ++a)
            if (members[a] < 0 || members[a] >= n || (a > grp_ptr[g] && members[a] <= members[a - 1]))
                return SIC_ERR_INVALID;  // positions in range, ascending within a group
    }
    SuffixGrids sg;
    sg.build(pts, n, dim, std::max<int64_t>(256, 4LL * n_cand), n_threads);
    std::vector<int32_t> cnt(n_grp, 0);
    parallel_for(n_grp, n_threads, 16, [&](int64_t g) {
        thread_local std::vector<KeyPos> buf;
        thread_local std::vector<int32_t> nb;
        const int64_t a = grp_ptr[g], b = grp_ptr[g + 1];
        const int m = (int)(b - a);
        nb.resize((size_t)n_cand + m);
        // nearest (to any member) points after the first member; the other members among
        // them are dropped (they enter every earlier member's column by themselves)
        int32_t got = knn_query(pts, n, dim, sg, members + a, m, members[a] + 1, n_cand + m - 1, nb.data(), buf);
        int32_t w = 0;
        int32_t* out = cand_idx + g * (int64_t)n_cand;
        for (int32_t q = 0; q < got && w < n_cand; ++q) {
            if (std::binary_search(members + a, members + b, (int64_t)nb[q])) continue;
            out[w++] = nb[q];
        }
        cnt[g] = w;
    });
    cand_ptr[0] = 0;
    for (int64_t g = 0; g < n_grp; ++g) {
        int64_t src = g * (int64_t)n_cand, dst = cand_ptr[g];
        if (dst != src) std::copy(cand_idx + src, cand_idx + src + cnt[g], cand_idx + dst);
        cand_ptr[g + 1] = dst + cnt[g];
    }
    return SIC_OK;
}

// Contiguous unit ranges of near-equal estimated cost for building one factor in slices.
extern "C" sic_status sic_prep_partition(const int64_t* cand_ptr, const int64_t* grp_ptr, int64_t n_units, int32_t k,
                                         int32_t max_cand, int32_t n_parts, int64_t* bounds) {
    if (!cand_ptr || !bounds || n_units < 0 || k < 0 || n_parts < 1) return SIC_ERR_INVALID;
    // running cost W[u] of units 0 .. u-1
    std::vector<double> W((size_t)n_units + 1, 0.0);
    const double kk = (double)k;
    for (int64_t u = 0; u < n_units; ++u) {
        int64_t c = cand_ptr[u + 1] - cand_ptr[u];
        if (c < 0) return SIC_ERR_INVALID;
        if (max_cand > 0 && c > max_cand) c = max_cand;
        const int64_t mi = grp_ptr ? grp_ptr[u + 1] - grp_ptr[u] : 1;
        if (mi < 1) return SIC_ERR_INVALID;
        const double m = (double)mi, C = (double)c, nn = kk + m;
        const double select = C * (kk * kk + kk * m + 0.5 * m * m);
        const double fill = nn * nn * nn / 6.0 + 0.5 * m * nn * nn;
        W[(size_t)u + 1] = W[(size_t)u] + select + 13.0 * fill;
    }
    const double total = W[(size_t)n_units];
    bounds[0] = 0;
    for (int32_t r = 1; r < n_parts; ++r) {
        // first u with W[u] >= r / n_parts of the total (the cut falls between units)
        const double target = total * (double)r / (double)n_parts;
        int64_t u = (int64_t)(std::lower_bound(W.begin(), W.end(), target) - W.begin());
        if (u > n_units) u = n_units;
        if (u < bounds[r - 1]) u = bounds[r - 1];
        bounds[r] = u;
    }
    bounds[n_parts] = n_units;
    return SIC_OK;
}
