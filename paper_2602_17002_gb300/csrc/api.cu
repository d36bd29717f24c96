// C ABI of libtlfe: mesh creation (validation, tile layout, reference
// precompute, colouring), the element operations, status handling.
// The Newton/CG step lives in newton.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <string>
#include <atomic>
#include <new>
#include <thread>
#include <vector>

#include "tlfe_elem.cuh"
#include "tlfe_fused.h"
#include "tlfe_internal.h"
#include "tlfe_mesh.h"

using namespace tlfe;

namespace tlfe {

static thread_local std::string g_err = "";

tlfe_status fail(tlfe_status st, const std::string &msg)
{
    g_err = msg;
    return st;
}

tlfe_status cuda_fail(cudaError_t e, const char *where)
{
    g_err = std::string(where) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? TLFE_E_OOM : TLFE_E_CUDA;
}

void *dalloc(tlfe_mesh *m, size_t bytes, cudaError_t *err)
{
    void *p = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
        *err = e;
        return nullptr;
    }
    m->allocs.push_back(p);
    m->device_bytes += (int64_t)bytes;
    return p;
}

}  // namespace tlfe

#define CK(call)                                                      \
    do {                                                              \
        cudaError_t e_ = (call);                                      \
        if (e_ != cudaSuccess) return tlfe::cuda_fail(e_, #call);     \
    } while (0)

#define CKA(ptr, bytes, m)                                            \
    do {                                                              \
        cudaError_t e_ = cudaSuccess;                                 \
        (ptr) = decltype(ptr)(tlfe::dalloc((m), (bytes), &e_));       \
        if (!(ptr)) return tlfe::cuda_fail(e_, "cudaMalloc " #ptr);   \
    } while (0)

// ---------------------------------------------------------------------------
// mesh creation
// ---------------------------------------------------------------------------

static bool valid_nq(int et, int nq)
{
    return (et == ET_T4 && nq == 1) || (et == ET_T10 && (nq == 4 || nq == 5)) || (et == ET_H8 && nq == 8) ||
           (et == ET_Q27 && nq == 27);
}

static tlfe_status validate(const tlfe_mesh_desc *d)
{
    if (!d) return fail(TLFE_E_INVALID, "desc is NULL");
    if (d->n_nodes <= 0 || !d->X_ref) return fail(TLFE_E_INVALID, "n_nodes must be > 0 and X_ref non-NULL");
    if (d->n_blocks <= 0 || !d->blocks) return fail(TLFE_E_INVALID, "n_blocks must be > 0 and blocks non-NULL");
    if (d->n_bodies <= 0 || !d->body_mat) return fail(TLFE_E_INVALID, "n_bodies must be > 0 and body_mat non-NULL");
    if (d->precision != TLFE_FP32 && d->precision != TLFE_FP64) return fail(TLFE_E_INVALID, "bad precision");
    if (d->scatter != TLFE_SCATTER_ATOMIC && d->scatter != TLFE_SCATTER_COLOR && d->scatter != TLFE_SCATTER_SORTED)
        return fail(TLFE_E_INVALID, "bad scatter mode");
    if (d->element_path != TLFE_PATH_AUTO && d->element_path != TLFE_PATH_SLAB && d->element_path != TLFE_PATH_AFFINE)
        return fail(TLFE_E_INVALID, "bad element path");
    if (d->patch_layout != TLFE_PATCH_BANKED && d->patch_layout != TLFE_PATCH_SORTED)
        return fail(TLFE_E_INVALID, "bad patch layout");
    for (int k = 0; k < 3 * d->n_nodes; ++k)
        if (!std::isfinite(d->X_ref[k])) return fail(TLFE_E_INVALID, "X_ref holds a non-finite value");
    for (int b = 0; b < d->n_bodies; ++b) {
        const tlfe_material &m = d->body_mat[b];
        if (m.model != TLFE_SVK && m.model != TLFE_NEOHOOKE && m.model != TLFE_MOONEY_RIVLIN)
            return fail(TLFE_E_INVALID, "bad material model");
        if (!std::isfinite(m.mu) || !std::isfinite(m.lambda) || !std::isfinite(m.mu_v) ||
            !std::isfinite(m.lambda_v) || !std::isfinite(m.rho) || m.mu_v < 0 || m.lambda_v < 0 || m.rho < 0)
            return fail(TLFE_E_INVALID, "bad material parameters");
        if (m.model == TLFE_MOONEY_RIVLIN && !std::isfinite(m.mu01))
            return fail(TLFE_E_INVALID, "bad Mooney-Rivlin mu01");
    }
    int64_t ne = 0;
    for (int bi = 0; bi < d->n_blocks; ++bi) {
        const tlfe_block &b = d->blocks[bi];
        if (b.type < 0 || b.type > 3) return fail(TLFE_E_INVALID, "bad element type");
        if (!valid_nq(b.type, b.n_qp)) return fail(TLFE_E_UNSUPPORTED, "unsupported quadrature size for the element type");
        if (b.n_elem < 0 || (b.n_elem > 0 && !b.conn)) return fail(TLFE_E_INVALID, "bad block element count / conn");
        const int npe = nodes_per_elem(b.type);
        for (int64_t k = 0; k < (int64_t)b.n_elem * npe; ++k)
            if (b.conn[k] < 0 || b.conn[k] >= d->n_nodes)
                return fail(TLFE_E_INVALID, "connectivity entry out of range in block " + std::to_string(bi));
        if (b.body)
            for (int k = 0; k < b.n_elem; ++k)
                if (b.body[k] < 0 || b.body[k] >= d->n_bodies)
                    return fail(TLFE_E_INVALID, "body id out of range in block " + std::to_string(bi));
        ne += b.n_elem;
    }
    if (ne <= 0 || ne > (int64_t)INT32_MAX / 2) return fail(TLFE_E_INVALID, "total element count out of range");
    if (d->elem_mu_lambda)
        for (int64_t k = 0; k < 2 * ne; ++k)
            if (!std::isfinite(d->elem_mu_lambda[k])) return fail(TLFE_E_INVALID, "elem_mu_lambda non-finite");
    return TLFE_OK;
}

// greedy-equivalent Jones-Plassmann colouring of one block on the device
static tlfe_status color_block(tlfe_mesh *m, const tlfe_block &b, uint64_t seed, std::vector<int32_t> &col,
                               cudaStream_t s)
{
    const int npe = nodes_per_elem(b.type);
    const int n = b.n_elem;
    // node -> incident elements (CSR) of this block
    std::vector<int32_t> off(m->n_nodes + 1, 0), inc((size_t)n * npe);
    for (int64_t k = 0; k < (int64_t)n * npe; ++k) off[b.conn[k] + 1]++;
    for (int k = 0; k < m->n_nodes; ++k) off[k + 1] += off[k];
    std::vector<int32_t> fill(m->n_nodes, 0);
    for (int e = 0; e < n; ++e)
        for (int i = 0; i < npe; ++i) {
            const int nd = b.conn[(int64_t)e * npe + i];
            inc[off[nd] + fill[nd]++] = e;
        }
    int32_t *d_conn, *d_off, *d_inc, *d_col;
    int *d_cnt;
    size_t bytes = sizeof(int32_t) * ((size_t)n * npe * 2 + m->n_nodes + 1 + n) + 2 * sizeof(int);
    char *buf = nullptr;
    CK(cudaMalloc(&buf, bytes));
    d_conn = (int32_t *)buf;
    d_inc = d_conn + (size_t)n * npe;
    d_off = d_inc + (size_t)n * npe;
    d_col = d_off + m->n_nodes + 1;
    d_cnt = (int *)(d_col + n);
    tlfe_status st = TLFE_OK;
    int h_cnt[2] = {n, 0};
    cudaError_t e = cudaMemcpyAsync(d_conn, b.conn, sizeof(int32_t) * n * npe, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_inc, inc.data(), sizeof(int32_t) * n * npe, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_off, off.data(), sizeof(int32_t) * (m->n_nodes + 1), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_col, 0xff, sizeof(int32_t) * n, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_cnt, h_cnt, sizeof(h_cnt), cudaMemcpyHostToDevice, s);
    // each round colours at least the highest-priority uncoloured element, so
    // n rounds always suffice; in practice a few dozen do
    for (int round = 0; e == cudaSuccess && round <= n; ++round) {
        e = launch_color_round(n, npe, d_conn, d_off, d_inc, nullptr, seed, 0, d_col, d_cnt, d_cnt + 1, s);
        if (e != cudaSuccess) break;
        e = cudaMemcpyAsync(h_cnt, d_cnt, sizeof(h_cnt), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess || h_cnt[0] == 0 || h_cnt[1]) break;
    }
    if (e != cudaSuccess) st = cuda_fail(e, "colouring");
    else if (h_cnt[1]) st = fail(TLFE_E_UNSUPPORTED, "more than 256 colours needed");
    else if (h_cnt[0] != 0) st = fail(TLFE_E_CUDA, "colouring did not finish");
    if (st == TLFE_OK) {
        col.resize(n);
        e = cudaMemcpy(col.data(), d_col, sizeof(int32_t) * n, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) st = cuda_fail(e, "colour download");
    }
    cudaFree(buf);
    return st;
}

template <typename R> static Mat<R> to_mat(const tlfe_material &s)
{
    Mat<R> m;
    m.model = s.model;
    m.mu = R(s.mu);
    m.lam = R(s.lambda);
    m.mu_v = R(s.mu_v);
    m.lam_v = R(s.lambda_v);
    m.rho = R(s.rho);
    m.mu01 = s.model == TLFE_MOONEY_RIVLIN ? R(s.mu01) : R(0);
    return m;
}

// 21 bits of x, y, z interleaved into one 63-bit Morton key
static uint64_t morton3(uint32_t x, uint32_t y, uint32_t z)
{
    auto spread = [](uint64_t v) {
        v &= 0x1FFFFF;
        v = (v | v << 32) & 0x1F00000000FFFFull;
        v = (v | v << 16) & 0x1F0000FF0000FFull;
        v = (v | v << 8) & 0x100F00F00F00F00Full;
        v = (v | v << 4) & 0x10C30C30C30C30C3ull;
        v = (v | v << 2) & 0x1249249249249249ull;
        return v;
    };
    return spread(x) | spread(y) << 1 | spread(z) << 2;
}

// unique nodes of the tiles of 32 consecutive elements of `order`: the sum
// over the tiles plus the tile count times the largest (the gather work, and
// the node patch that sets the shared memory of every warp)
static int64_t tile_node_cost(const tlfe_mesh_desc *d, const tlfe_block &b, const std::vector<int32_t> &order)
{
    const int npe = nodes_per_elem(b.type);
    std::vector<int32_t> stamp(d->n_nodes, -1);
    int64_t total = 0, umax = 0, u = 0;
    for (size_t k = 0; k < order.size(); ++k) {
        const int tile = (int)(k / TILE);
        if (k % TILE == 0) u = 0;
        for (int i = 0; i < npe; ++i) {
            const int32_t n = b.conn[(int64_t)order[k] * npe + i];
            if (stamp[n] != tile) {
                stamp[n] = tile;
                ++total;
                ++u;
            }
        }
        umax = std::max(umax, u);
    }
    return total + (int64_t)((order.size() + TILE - 1) / TILE) * umax;
}

// Element order of the tiles. Candidates: the input order, and orders by
// body, then along a Morton curve of the element centroids, then by element
// index. The curve quantises each body's centroids on a cubic grid of step
// f h, h = (bounding-box volume / elements)^(1/3), for f = 1 (one brick per
// cell), 5^(1/3) and 6^(1/3) (five or six tetrahedra per cell) and 2, so that
// on a structured mesh the grid cells are the mesh cells and 32 consecutive
// elements form a compact block of cells; bodies that overlap in space are
// not interleaved. A curve order replaces the input order only when it cuts
// tile_node_cost by 15 % or more: on the beam of Kuhn tetrahedra numbered
// cell by cell its 5 % saving measured slower than the input order, while on
// bricks numbered row by row it saves about 30 % and measured 25 % faster.
static std::vector<int32_t> locality_order(const tlfe_mesh_desc *d, const tlfe_block &b)
{
    const int npe = nodes_per_elem(b.type);
    const int n = b.n_elem;
    std::vector<int32_t> best(n);
    std::iota(best.begin(), best.end(), 0);
    if (n <= TILE) return best;
    const int64_t ident_cost = tile_node_cost(d, b, best);
    int64_t best_cost = ident_cost;
    // per body: node bounding box and element count
    auto body_of = [&](int e) { return b.body ? b.body[e] : 0; };
    int nb = 0;
    for (int e = 0; e < n; ++e) nb = std::max(nb, body_of(e) + 1);
    std::vector<double> lo((size_t)nb * 3, INFINITY), hi((size_t)nb * 3, -INFINITY);
    std::vector<int64_t> cnt(nb, 0);
    std::vector<double> c((size_t)n * 3, 0.0);
    for (int e = 0; e < n; ++e) {
        const int bo = body_of(e);
        ++cnt[bo];
        for (int a = 0; a < 3; ++a) {
            double sum = 0.0;
            for (int i = 0; i < npe; ++i) {
                const double x = d->X_ref[(size_t)b.conn[(int64_t)e * npe + i] * 3 + a];
                sum += x;
                lo[(size_t)bo * 3 + a] = std::min(lo[(size_t)bo * 3 + a], x);
                hi[(size_t)bo * 3 + a] = std::max(hi[(size_t)bo * 3 + a], x);
            }
            c[(size_t)e * 3 + a] = sum / npe;
        }
    }
    std::vector<double> h0(nb, 0.0);
    for (int bo = 0; bo < nb; ++bo) {
        if (cnt[bo] == 0) continue;
        double vol = 1.0, ext = 0.0;
        for (int a = 0; a < 3; ++a) {
            vol *= hi[(size_t)bo * 3 + a] - lo[(size_t)bo * 3 + a];
            ext = std::max(ext, hi[(size_t)bo * 3 + a] - lo[(size_t)bo * 3 + a]);
        }
        h0[bo] = vol > 0.0 ? std::cbrt(vol / (double)cnt[bo]) : ext / std::cbrt((double)cnt[bo]);
    }
    struct Key {
        int32_t body;
        uint64_t code;
        int32_t e;
        bool operator<(const Key &o) const
        {
            return body != o.body ? body < o.body : (code != o.code ? code < o.code : e < o.e);
        }
    };
    std::vector<Key> key(n);
    std::vector<int32_t> order(n);
    for (double f : {1.0, std::cbrt(5.0), std::cbrt(6.0), 2.0}) {
        for (int e = 0; e < n; ++e) {
            const int bo = body_of(e);
            const double h = f * h0[bo];
            uint32_t q[3] = {0, 0, 0};
            for (int a = 0; a < 3; ++a) {
                const double v = h > 0.0 ? std::floor((c[(size_t)e * 3 + a] - lo[(size_t)bo * 3 + a]) / h) : 0.0;
                q[a] = (uint32_t)std::min(std::max(v, 0.0), (double)((1u << 21) - 1));
            }
            key[e] = {bo, morton3(q[0], q[1], q[2]), e};
        }
        std::sort(key.begin(), key.end());
        for (int e = 0; e < n; ++e) order[e] = key[e].e;
        const int64_t cost = tile_node_cost(d, b, order);
        if (cost < best_cost && cost <= ident_cost - ident_cost * 15 / 100) {
            best_cost = cost;
            best = order;
        }
    }
    return best;
}

// Shared-memory passes of the node-patch loads of one tile. The FP32 element
// kernels read a node's 48-byte patch record in 16-byte loads, and the 8
// lanes of a quarter warp (one pass of a 16-byte load) all read the record of
// the same element-local node i of their elements: record s starts in 16-byte
// bank group 3 s mod 8, so distinct records whose slots agree mod 8 are read
// in separate passes (equal records are one broadcast). `li` holds [npe][32]
// slots, `valid` the lanes that hold an element; returns the passes summed
// over (i, quarter) and adds the loads to *loads.
static int64_t patch_tile_passes(int npe, const uint16_t *li, const bool *valid, int64_t *loads)
{
    int64_t passes = 0;
    for (int i = 0; i < npe; ++i)
        for (int q = 0; q < TILE / 8; ++q) {
            int seen[8], ns = 0, mult[8] = {0, 0, 0, 0, 0, 0, 0, 0};
            for (int l = q * 8; l < q * 8 + 8; ++l) {
                if (!valid[l]) continue;
                const int sl = li[i * TILE + l];
                bool dup = false;
                for (int k = 0; k < ns; ++k) dup = dup || seen[k] == sl;
                if (dup) continue;
                seen[ns++] = sl;
                ++mult[sl & 7];
            }
            if (ns == 0) continue;
            ++*loads;
            passes += *std::max_element(mult, mult + 8);
        }
    return passes;
}

// Patch slots of a tile's U unique nodes (TLFE_PATCH_BANKED): nodes read
// together by a quarter warp (see patch_tile_passes) get distinct slots mod 8.
// The gather and the scatter walk the list 32 entries per warp instruction,
// so each run of 32 consecutive nodes in ascending id keeps its entries (its
// nodes only change places inside the run): the warp's global accesses touch
// the same sectors as in ascending order. A run of n nodes owns the slots
// 32 j .. 32 j + n - 1, of which those with residue c (mod 8) number
// (n - c + 7) / 8 for c < n; inside that limit this colours the conflict
// graph with the 8 residues: nodes by decreasing conflict count, each onto
// the residue its already placed neighbours use least among those its run
// still has slots of (ties: the most free slots, then the lowest residue);
// then, while some node gains, a move to a residue with a free slot or a
// swap with a node of another residue in its run. Node k of run j gets slot
// 32 j + 8 r + c, c its residue and r its rank among the run's nodes of that
// residue: a permutation of 0 .. U - 1 (no holes). `pos` holds [npe][32]
// indices into the sorted list.
static void patch_slots(int U, int npe, const uint16_t *pos, const bool *valid, std::vector<uint16_t> &slot)
{
    // the loads: distinct nodes of each (i, quarter)
    static thread_local std::vector<int> gk, deg, adj, fill, col, order, cnt, cap;
    const int n_loads = npe * (TILE / 8);
    gk.assign((size_t)n_loads * 9, 0);
    for (int g = 0; g < n_loads; ++g) {
        const int i = g / (TILE / 8), q = g % (TILE / 8);
        int *G = gk.data() + (size_t)g * 9, ng = 0;
        for (int l = q * 8; l < q * 8 + 8; ++l) {
            if (!valid[l]) continue;
            const int k = pos[i * TILE + l];
            bool dup = false;
            for (int j = 0; j < ng; ++j) dup = dup || G[1 + j] == k;
            if (!dup) G[1 + ng++] = k;
        }
        G[0] = ng;
    }
    // conflict lists (a pair sharing several loads appears once per load)
    deg.assign(U + 1, 0);
    for (int g = 0; g < n_loads; ++g) {
        const int *G = gk.data() + (size_t)g * 9;
        for (int a = 0; a < G[0]; ++a) deg[G[1 + a] + 1] += G[0] - 1;
    }
    for (int k = 0; k < U; ++k) deg[k + 1] += deg[k];
    adj.resize(deg[U]);
    fill.assign(deg.begin(), deg.end() - 1);
    for (int g = 0; g < n_loads; ++g) {
        const int *G = gk.data() + (size_t)g * 9;
        for (int a = 0; a < G[0]; ++a)
            for (int b = 0; b < G[0]; ++b)
                if (a != b) adj[fill[G[1 + a]]++] = G[1 + b];
    }
    // runs of 32 and their slots per residue
    const int n_runs = (U + 31) / 32;
    cnt.assign((size_t)n_runs * 8, 0);
    cap.resize((size_t)n_runs * 8);
    for (int j = 0; j < n_runs; ++j) {
        const int n = std::min(32, U - 32 * j);
        for (int c = 0; c < 8; ++c) cap[(size_t)j * 8 + c] = c < n ? (n - c + 7) / 8 : 0;
    }
    col.assign(U, -1);
    order.resize(U);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return deg[a + 1] - deg[a] > deg[b + 1] - deg[b]; });
    auto conflicts = [&](int a, int *c8) {
        for (int c = 0; c < 8; ++c) c8[c] = 0;
        for (int j = deg[a]; j < deg[a + 1]; ++j)
            if (col[adj[j]] >= 0) ++c8[col[adj[j]]];
    };
    for (int a : order) {
        int c8[8], best = -1;
        const int *n8 = cnt.data() + (size_t)(a / 32) * 8;
        const int *k8 = cap.data() + (size_t)(a / 32) * 8;
        conflicts(a, c8);
        for (int c = 0; c < 8; ++c) {
            if (n8[c] >= k8[c]) continue;
            if (best < 0 || c8[c] < c8[best] || (c8[c] == c8[best] && k8[c] - n8[c] > k8[best] - n8[best])) best = c;
        }
        col[a] = best;
        ++cnt[(size_t)(a / 32) * 8 + best];
    }
    for (int pass = 0; pass < 8; ++pass) {
        bool changed = false;
        for (int a = 0; a < U; ++a) {
            int c8[8];
            conflicts(a, c8);
            const int ca = col[a], j = a / 32;
            if (c8[ca] == 0) continue;
            int *n8 = cnt.data() + (size_t)j * 8;
            const int *k8 = cap.data() + (size_t)j * 8;
            int best = ca;
            for (int c = 0; c < 8; ++c)
                if (c != ca && n8[c] < k8[c] && c8[c] < c8[best]) best = c;
            if (best != ca) {
                --n8[ca];
                ++n8[best];
                col[a] = best;
                changed = true;
                continue;
            }
            // swap with the node b of the run that lowers the conflicts of
            // a and b the most (entries of a and b on each other drop out)
            int gain = 0, swap_with = -1;
            for (int b = 32 * j; b < std::min(U, 32 * j + 32); ++b) {
                const int cb = col[b];
                if (cb == ca) continue;
                int d8[8], ab = 0;
                conflicts(b, d8);
                for (int e = deg[a]; e < deg[a + 1]; ++e) ab += adj[e] == b;
                const int g = (c8[ca] + d8[cb]) - ((c8[cb] - ab) + (d8[ca] - ab));
                if (g > gain) {
                    gain = g;
                    swap_with = b;
                }
            }
            if (swap_with >= 0) {
                std::swap(col[a], col[swap_with]);
                changed = true;
            }
        }
        if (!changed) break;
    }
    slot.assign(U, 0);
    for (int j = 0; j < n_runs; ++j) {
        int rank[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int a = 32 * j; a < std::min(U, 32 * j + 32); ++a)
            slot[a] = (uint16_t)(32 * j + 8 * rank[col[a]]++ + col[a]);
    }
}

static tlfe_status build_block(tlfe_mesh *m, const tlfe_mesh_desc *d, int bi, int elem_base, cudaStream_t s)
{
    const tlfe_block &b = d->blocks[bi];
    BlockStore &B = m->blocks[bi];
    B.et = b.type;
    B.nq = b.n_qp;
    B.npe = nodes_per_elem(b.type);
    B.n_elem = b.n_elem;
    B.elem_base = elem_base;
    const int npe = B.npe;

    // the material of block element k: its body's
    const bool have_body = b.body != nullptr && b.n_elem > 0;
    auto mat_of = [&](int k) -> const tlfe_material & { return d->body_mat[have_body ? b.body[k] : 0]; };

    // element order inside the layout: the locality order, then grouped by
    // colour (colour mode) and by elastic law, keeping that order inside each
    // group. Every group starts a new tile and is launched as its own pass,
    // so that a pass has one law and runs that law's specialised kernel.
    std::vector<int32_t> order = locality_order(d, b);
    B.n_colors = 0;
    const bool colour_mode = d->scatter == TLFE_SCATTER_COLOR;
    if (colour_mode && b.n_elem > 0) {
        std::vector<int32_t> col;
        tlfe_status st = color_block(m, b, d->color_seed, col, s);
        if (st != TLFE_OK) return st;
        B.colors = col;
        B.n_colors = *std::max_element(col.begin(), col.end()) + 1;
    }
    auto group = [&](int k) -> int64_t { return (int64_t)(colour_mode ? B.colors[k] : 0) * 4 + mat_of(k).model; };
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return group(a) < group(c); });
    std::vector<int32_t> eid;
    B.color_tile_off.assign(1, 0);
    B.pass_model.clear();
    B.pass_visc.clear();
    for (size_t k = 0; k < order.size();) {
        const int64_t g = group(order[k]);
        B.pass_model.push_back(mat_of(order[k]).model);
        bool damped = false;
        for (; k < order.size() && group(order[k]) == g; ++k) {
            const tlfe_material &mm = mat_of(order[k]);
            damped = damped || mm.mu_v != 0.0 || mm.lambda_v != 0.0;
            eid.push_back(elem_base + order[k]);
        }
        while (eid.size() % TILE) eid.push_back(-1);
        B.color_tile_off.push_back((int)(eid.size() / TILE));
        B.pass_visc.push_back(damped);
    }
    B.n_tiles = (int)(eid.size() / TILE);

    // per tile: its node list (the unique nodes, in ascending id or, in the
    // banked patch layout, permuted to their patch slots), (element, node) ->
    // list index, and for each slot i*32 + lane its position in the
    // node-grouped order (the positions of list entry kk are [soff[kk],
    // soff[kk + 1])). Tiles are independent:
    // batches of them are built on the host's cores, then appended in order.
    std::vector<int32_t> toff(B.n_tiles + 1, 0), tnodes;
    std::vector<uint16_t> lidx((size_t)B.n_tiles * npe * TILE, 0);
    std::vector<uint16_t> nsl((size_t)B.n_tiles * npe * TILE, 0xFFFF), soff;
    soff.reserve((size_t)B.n_tiles * (npe * 12 + 1));
    tnodes.reserve((size_t)B.n_tiles * npe * 12);
    B.umax = 1;
    B.patch_loads = B.patch_passes = 0;
    struct TileList {
        std::vector<int32_t> nodes;
        std::vector<uint16_t> soff;
        int64_t loads = 0, passes = 0;
    };
    const bool banked = d->patch_layout == TLFE_PATCH_BANKED;
    auto build_tile = [&](int t, TileList &o) {
        static thread_local std::vector<int32_t> ulist;
        static thread_local std::vector<uint16_t> slot;
        static thread_local std::vector<int> cnt;
        std::vector<int32_t> &tmp = o.nodes;
        tmp.clear();
        bool valid[TILE];
        for (int l = 0; l < TILE; ++l) {
            const int e = eid[(size_t)t * TILE + l];
            valid[l] = e >= 0;
            if (e < 0) continue;
            for (int i = 0; i < npe; ++i) tmp.push_back(b.conn[(int64_t)(e - elem_base) * npe + i]);
        }
        std::sort(tmp.begin(), tmp.end());
        tmp.erase(std::unique(tmp.begin(), tmp.end()), tmp.end());
        uint16_t *lt = lidx.data() + (size_t)t * npe * TILE;
        for (int l = 0; l < TILE; ++l) {
            if (!valid[l]) continue;
            const int e = eid[(size_t)t * TILE + l];
            for (int i = 0; i < npe; ++i) {
                const int nd = b.conn[(int64_t)(e - elem_base) * npe + i];
                lt[i * TILE + l] = (uint16_t)(std::lower_bound(tmp.begin(), tmp.end(), nd) - tmp.begin());
            }
        }
        // the banked layout moves node k of the sorted list to slot[k] (a
        // permutation of the list)
        if (banked && !tmp.empty()) {
            patch_slots((int)tmp.size(), npe, lt, valid, slot);
            for (int k = 0; k < npe * TILE; ++k) lt[k] = valid[k % TILE] ? slot[lt[k]] : slot[0];
            ulist.resize(tmp.size());
            for (size_t k = 0; k < tmp.size(); ++k) ulist[slot[k]] = tmp[k];
            tmp.swap(ulist);
        }
        o.loads = 0;
        o.passes = patch_tile_passes(npe, lt, valid, &o.loads);
        const int U = (int)tmp.size();
        cnt.assign(U + 1, 0);
        for (int l = 0; l < TILE; ++l)
            if (valid[l])
                for (int i = 0; i < npe; ++i) cnt[lt[i * TILE + l] + 1]++;
        for (int k = 0; k < U; ++k) cnt[k + 1] += cnt[k];
        o.soff.assign(cnt.begin(), cnt.end());
        uint16_t *nt = nsl.data() + (size_t)t * npe * TILE;
        for (int i = 0; i < npe; ++i)
            for (int l = 0; l < TILE; ++l)
                if (valid[l]) nt[i * TILE + l] = (uint16_t)(cnt[lt[i * TILE + l]]++);
    };
    {
        constexpr int BATCH = 8192;
        const int nthr = (int)std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
        std::vector<TileList> out((size_t)std::min(B.n_tiles, BATCH));
        for (int t0 = 0; t0 < B.n_tiles; t0 += BATCH) {
            const int t1 = std::min(B.n_tiles, t0 + BATCH);
            // a host allocation failing in a worker is passed on after the join
            std::atomic<bool> failed(false);
            auto worker = [&](int w, int nw) {
                try {
                    for (int t = t0 + w; t < t1 && !failed.load(); t += nw) build_tile(t, out[t - t0]);
                } catch (...) {
                    failed.store(true);
                }
            };
            if (nthr == 1 || t1 - t0 < 256) {
                worker(0, 1);
            } else {
                std::vector<std::thread> pool;
                std::vector<int> here;  // shares whose thread could not be started run on this one
                for (int w = 0; w < nthr; ++w) {
                    try {
                        pool.emplace_back(worker, w, nthr);
                    } catch (...) {
                        here.push_back(w);
                    }
                }
                for (int w : here) worker(w, nthr);
                for (auto &th : pool) th.join();
            }
            if (failed.load()) throw std::bad_alloc();
            for (int t = t0; t < t1; ++t) {
                const TileList &o = out[t - t0];
                tnodes.insert(tnodes.end(), o.nodes.begin(), o.nodes.end());
                soff.insert(soff.end(), o.soff.begin(), o.soff.end());
                toff[t + 1] = (int32_t)tnodes.size();
                B.umax = std::max(B.umax, (int)o.nodes.size());
                B.patch_loads += o.loads;
                B.patch_passes += o.passes;
            }
        }
    }
    B.n_unique = (int64_t)tnodes.size();

    // one fixed-size metadata record per tile, fetched by one bulk copy:
    //   [U, P, 0, 0 | eid[32] | node ids[umaxp] | lidx[npe][32] | position[npe*32] | soff[soffp]]
    // with P the tile's first partial-sum position (sorted scatter)
    const int64_t part_base = (int64_t)m->h_part_node.size();
    const int umaxp = (B.umax + 3) / 4 * 4;
    const int soffp = (B.umax + 1 + 7) / 8 * 8;
    B.meta_bytes = 16 + 4 * TILE + 4 * umaxp + 2 * 2 * npe * TILE + 2 * soffp;
    B.meta_umaxp = umaxp;
    std::vector<unsigned char> meta((size_t)B.n_tiles * B.meta_bytes, 0);
    {
        size_t so = 0;
        for (int t = 0; t < B.n_tiles; ++t) {
            unsigned char *r = meta.data() + (size_t)t * B.meta_bytes;
            const int U = toff[t + 1] - toff[t];
            int32_t *hdr = (int32_t *)r;
            hdr[0] = U;
            hdr[1] = (int32_t)std::min<int64_t>(INT32_MAX, part_base + toff[t]);
            memcpy(r + 16, eid.data() + (size_t)t * TILE, 4 * TILE);
            memcpy(r + 16 + 4 * TILE, tnodes.data() + toff[t], 4 * (size_t)U);
            unsigned char *q = r + 16 + 4 * TILE + 4 * umaxp;
            memcpy(q, lidx.data() + (size_t)t * npe * TILE, 2 * (size_t)npe * TILE);
            memcpy(q + 2 * npe * TILE, nsl.data() + (size_t)t * npe * TILE, 2 * (size_t)npe * TILE);
            memcpy(q + 4 * npe * TILE, soff.data() + so, 2 * (size_t)(U + 1));
            so += U + 1;
        }
    }

    // materials: uniform when all elements of the block share one body
    const int body0 = have_body ? b.body[0] : 0;
    bool uniform = true;
    if (have_body)
        for (int k = 0; k < b.n_elem; ++k)
            if (b.body[k] != body0) uniform = false;
    B.uniform_body = uniform ? body0 : -1;
    B.visc = false;
    B.model = b.n_elem > 0 ? d->body_mat[body0].model : -1;
    for (int k = 0; k < b.n_elem; ++k) {
        const tlfe_material &mm = d->body_mat[have_body ? b.body[k] : 0];
        if (mm.mu_v != 0.0 || mm.lambda_v != 0.0) B.visc = true;
        if (mm.model != B.model) B.model = -1;
        if (uniform) break;
    }
    const size_t rs = m->precision == TLFE_FP32 ? 4 : 8;
    const size_t nslot = (size_t)B.n_tiles * TILE;
    CKA(B.d_eid, sizeof(int32_t) * nslot, m);
    CKA(B.d_toff, sizeof(int32_t) * (B.n_tiles + 1), m);
    CKA(B.d_tnodes, sizeof(int32_t) * tnodes.size(), m);
    CKA(B.d_lidx, sizeof(uint16_t) * lidx.size(), m);
    CKA(B.d_meta, meta.size(), m);
    CKA(B.d_evol, rs * nslot, m);
    CK(cudaMemcpyAsync(B.d_eid, eid.data(), sizeof(int32_t) * nslot, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(B.d_toff, toff.data(), sizeof(int32_t) * toff.size(), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(B.d_tnodes, tnodes.data(), sizeof(int32_t) * tnodes.size(), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(B.d_lidx, lidx.data(), sizeof(uint16_t) * lidx.size(), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(B.d_meta, meta.data(), meta.size(), cudaMemcpyHostToDevice, s));
    // the host vectors are released below, before the copies have run: wait
    CK(cudaStreamSynchronize(s));
    B.d_emat = nullptr;
    if (!uniform) {
        std::vector<int32_t> em(nslot, 0);
        for (size_t k = 0; k < nslot; ++k)
            if (eid[k] >= 0) em[k] = b.body[eid[k] - elem_base];
        CKA(B.d_emat, sizeof(int32_t) * nslot, m);
        CK(cudaMemcpyAsync(B.d_emat, em.data(), sizeof(int32_t) * nslot, cudaMemcpyHostToDevice, s));
    }
    B.d_elam = nullptr;
    if (d->elem_mu_lambda) {
        CKA(B.d_elam, rs * nslot * 2, m);
        std::vector<double> el(nslot * 2, 0.0);
        for (int t = 0; t < B.n_tiles; ++t)
            for (int l = 0; l < TILE; ++l) {
                const int e = eid[(size_t)t * TILE + l];
                if (e < 0) continue;
                el[((size_t)t * 2 + 0) * TILE + l] = d->elem_mu_lambda[(size_t)e * 2 + 0];
                el[((size_t)t * 2 + 1) * TILE + l] = d->elem_mu_lambda[(size_t)e * 2 + 1];
            }
        if (m->precision == TLFE_FP32) {
            std::vector<float> ef(el.begin(), el.end());
            CK(cudaMemcpy(B.d_elam, ef.data(), 4 * ef.size(), cudaMemcpyHostToDevice));
        } else {
            CK(cudaMemcpy(B.d_elam, el.data(), 8 * el.size(), cudaMemcpyHostToDevice));
        }
    }
    // reference precompute (Sec. 6) on the device: first J^{-1}, det J and the
    // affine test per element; then, for blocks on the slab path, the
    // per-point h_i and w_q J_p
    // the block connectivity stays on the device (external loads use it)
    CKA(B.d_conn, sizeof(int32_t) * std::max<size_t>(1, (size_t)b.n_elem * npe), m);
    int32_t *d_conn = B.d_conn;
    int *d_aflag = nullptr;
    CK(cudaMalloc(&d_aflag, sizeof(int)));
    const int one = 1;
    int aflag = 0;
    cudaError_t e = cudaSuccess;
    if (d->element_path != TLFE_PATH_SLAB) {
        e = cudaMalloc(&B.d_aff, rs * nslot * AFF_ROWS);
        if (e == cudaSuccess) {
            m->allocs.push_back(B.d_aff);
            m->device_bytes += (int64_t)(rs * nslot * AFF_ROWS);
        }
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_conn, b.conn, sizeof(int32_t) * b.n_elem * npe, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_aflag, &one, sizeof(int), cudaMemcpyHostToDevice, s);
    void *aff_out = B.d_aff;
    if (e == cudaSuccess && !aff_out) {  // slab path only: the affine test still runs, into scratch
        e = cudaMalloc(&aff_out, std::max<size_t>(16, rs * nslot * AFF_ROWS));
    }
    if (e == cudaSuccess)
        e = launch_precompute_affine(B.et, m->precision, B.n_tiles, B.d_eid, d_conn, elem_base, m->d_X, aff_out,
                                     B.d_evol, d_aflag, m->d_status, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&aflag, d_aflag, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (aff_out != B.d_aff) cudaFree(aff_out);
    B.affine = aflag != 0 && b.n_elem > 0;
    if (e == cudaSuccess && d->element_path == TLFE_PATH_AFFINE && !B.affine && b.n_elem > 0) {
        cudaFree(d_aflag);
        return fail(TLFE_E_UNSUPPORTED, "element_path = TLFE_PATH_AFFINE but block " + std::to_string(bi) +
                                            " has non-affine elements");
    }
    B.use_affine = B.affine && d->element_path != TLFE_PATH_SLAB;
    if (e == cudaSuccess && !B.use_affine) {
        e = cudaMalloc(&B.d_slab, rs * nslot * B.nq * (npe * 3 + 1));
        if (e == cudaSuccess) {
            m->allocs.push_back(B.d_slab);
            m->device_bytes += (int64_t)(rs * nslot * B.nq * (npe * 3 + 1));
            e = cudaMemcpyAsync(d_aflag, &one, sizeof(int), cudaMemcpyHostToDevice, s);
        }
        if (e == cudaSuccess)
            e = launch_precompute(B.et, B.nq, m->precision, B.n_tiles, B.d_eid, d_conn, elem_base, m->d_X,
                                  B.d_slab, B.d_evol, d_aflag, m->d_status, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    cudaFree(d_aflag);
    if (e != cudaSuccess) return cuda_fail(e, "reference precompute");

    // sorted scatter: the node of each of this block's partial-sum positions,
    // in the order the kernels store them (tile node lists, or 27 per slot on
    // the warp-per-element path)
    if (d->scatter == TLFE_SCATTER_SORTED) {
        std::vector<int32_t> &pn = m->h_part_node;
        B.part_base = part_base;
        if (wpe_path(B.et, B.use_affine)) {
            for (size_t k = 0; k < eid.size(); ++k)
                for (int i = 0; i < npe; ++i)
                    pn.push_back(eid[k] < 0 ? -1 : b.conn[(int64_t)(eid[k] - elem_base) * npe + i]);
        } else {
            pn.insert(pn.end(), tnodes.begin(), tnodes.end());
        }
        if (pn.size() > (size_t)INT32_MAX)
            return fail(TLFE_E_UNSUPPORTED, "sorted scatter: more than 2^31 partial sums");
    }
    return TLFE_OK;
}

// Work items of the fused launch: the passes the fused kernels cover (FP32,
// atomic or sorted scatter, affine T4 / T10 / H8 tile blocks), when there are
// at least two. Each pass is cut into runs of tiles of about equal work
// (quadrature points x nodes of FUSED_ITEM_COST per run); the items are
// listed longest first: the passes in decreasing work per tile, each in tile
// order (neighbouring runs share nodes through L2), then the shorter
// remainder runs in decreasing length, so that light items fill the tail.
constexpr int FUSED_ITEM_COST = 400;

static tlfe_status build_fused_plan(tlfe_mesh *m)
{
    if (m->precision != TLFE_FP32 || m->scatter == TLFE_SCATTER_COLOR) return TLFE_OK;
    std::vector<std::pair<int, int>> passes;
    std::vector<bool> covered(m->blocks.size(), false);
    for (int bi = 0; bi < (int)m->blocks.size(); ++bi) {
        const BlockStore &B = m->blocks[bi];
        if (B.n_elem == 0 || !B.use_affine || wpe_path(B.et, true) || fused_code(B.et, B.nq) < 0) continue;
        covered[bi] = true;
        for (int c = 0; c + 1 < (int)B.color_tile_off.size(); ++c)
            if (B.color_tile_off[c + 1] > B.color_tile_off[c]) passes.emplace_back(bi, c);
    }
    if (passes.size() < 2 || passes.size() > (size_t)FUSED_MAXP) return TLFE_OK;
    auto tile_cost = [&](int bi) { return m->blocks[bi].nq * m->blocks[bi].npe; };
    std::vector<int> order(passes.size());
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return tile_cost(passes[a].first) > tile_cost(passes[b].first); });
    std::vector<int4> full, rest;
    for (int k : order) {
        const BlockStore &B = m->blocks[passes[k].first];
        const int c = passes[k].second;
        const int per = std::max(1, std::min(1024, FUSED_ITEM_COST / tile_cost(passes[k].first)));
        for (int t = B.color_tile_off[c]; t < B.color_tile_off[c + 1]; t += per) {
            const int te = std::min(t + per, B.color_tile_off[c + 1]);
            (te - t == per ? full : rest).push_back(make_int4(k, t, te, 0));
        }
    }
    std::stable_sort(rest.begin(), rest.end(), [&](const int4 &a, const int4 &b) {
        return (int64_t)(a.z - a.y) * tile_cost(passes[a.x].first) > (int64_t)(b.z - b.y) * tile_cost(passes[b.x].first);
    });
    full.insert(full.end(), rest.begin(), rest.end());
    FusedPlan *fp = new FusedPlan();
    m->fused = fp;
    fp->passes = passes;
    fp->covered = covered;
    fp->n_items = (int)full.size();
    CKA(fp->d_items, sizeof(int4) * full.size(), m);
    CKA(fp->d_counter, sizeof(int) * 4, m);
    CK(cudaMemcpy(fp->d_items, full.data(), sizeof(int4) * full.size(), cudaMemcpyHostToDevice));
    for (int o = 0; o < 2; ++o) {
        size_t w = 0;
        for (auto &pc : passes) {
            const BlockStore &B = m->blocks[pc.first];
            const int code = fused_code(B.et, B.nq);
            w = std::max(w, o == 0 ? fused_warp_region<float, OP_FORCE>(code, B.umax, B.meta_bytes)
                                   : fused_warp_region<float, OP_MATVEC>(code, B.umax, B.meta_bytes));
        }
        fp->wreg[o] = w;
    }
    return TLFE_OK;
}

static tlfe_status create_mesh(const tlfe_mesh_desc *desc, cudaStream_t s, tlfe_mesh **out, tlfe_mesh **held);

// Host allocations (the mesh's host tables, the tile lists of a large batch)
// can fail; the exception does not cross the C ABI: the handle under
// construction is released and TLFE_E_OOM returned.
extern "C" tlfe_status tlfe_create_mesh(const tlfe_mesh_desc *desc, void *stream, tlfe_mesh **out)
{
    TLFE_TRACE("tlfe_create_mesh");
    if (!out) return fail(TLFE_E_INVALID, "out is NULL");
    *out = nullptr;
    tlfe_mesh *held = nullptr;  // the handle under construction, until create_mesh releases it itself
    tlfe_status st;
    try {
        st = create_mesh(desc, (cudaStream_t)stream, out, &held);
    } catch (const std::exception &ex) {
        st = fail(TLFE_E_OOM, std::string("host allocation failed while building the mesh (") + ex.what() + ")");
    }
    if (st != TLFE_OK) {
        if (held) tlfe_destroy_mesh(held);
        *out = nullptr;
    }
    return st;
}

static tlfe_status create_mesh(const tlfe_mesh_desc *desc, cudaStream_t s, tlfe_mesh **out, tlfe_mesh **held)
{
    tlfe_status st = validate(desc);
    if (st != TLFE_OK) return st;
    tlfe_mesh *m = new tlfe_mesh();
    *held = m;
    CK(cudaGetDevice(&m->device));
    CK(cudaDeviceGetAttribute(&m->n_sm, cudaDevAttrMultiProcessorCount, m->device));
    m->precision = desc->precision;
    m->scatter = desc->scatter;
    m->n_nodes = desc->n_nodes;
    m->n_bodies = desc->n_bodies;
    m->h_mats.assign(desc->body_mat, desc->body_mat + desc->n_bodies);
    m->blocks.resize(desc->n_blocks);
    m->color_seed = desc->color_seed;
    m->element_path = desc->element_path;
    m->patch_layout = desc->patch_layout;
    m->h_X.assign(desc->X_ref, desc->X_ref + 3 * (size_t)desc->n_nodes);
    m->node_body.assign(desc->n_nodes, -1);
    {
        int64_t ne = 0;
        for (int bi = 0; bi < desc->n_blocks; ++bi) {
            const tlfe_block &b = desc->blocks[bi];
            const int npe = nodes_per_elem(b.type);
            m->h_conn.emplace_back(b.conn, b.conn + (size_t)b.n_elem * npe);
            if (b.body) m->h_body.emplace_back(b.body, b.body + b.n_elem);
            else m->h_body.emplace_back((size_t)b.n_elem, 0);
            m->h_blocks.push_back(b);
            for (int e = 0; e < b.n_elem; ++e)
                for (int i = 0; i < npe; ++i) m->node_body[b.conn[(size_t)e * npe + i]] = m->h_body.back()[e];
            ne += b.n_elem;
        }
        if (desc->elem_mu_lambda) m->h_elam.assign(desc->elem_mu_lambda, desc->elem_mu_lambda + 2 * ne);
    }
    auto bail = [&](tlfe_status e) {
        *held = nullptr;
        tlfe_destroy_mesh(m);
        return e;
    };
#define CKM(call)                                                            \
    do {                                                                     \
        cudaError_t e_ = (call);                                             \
        if (e_ != cudaSuccess) return bail(tlfe::cuda_fail(e_, #call));      \
    } while (0)
    cudaError_t ae = cudaSuccess;
    m->d_status = (int *)dalloc(m, sizeof(int) * ST_COUNT, &ae);
    m->d_X = (double *)dalloc(m, sizeof(double) * 3 * m->n_nodes, &ae);
    m->d_mats_f = (Mat<float> *)dalloc(m, sizeof(Mat<float>) * m->n_bodies, &ae);
    m->d_mats_d = (Mat<double> *)dalloc(m, sizeof(Mat<double>) * m->n_bodies, &ae);
    if (ae != cudaSuccess) return bail(cuda_fail(ae, "cudaMalloc"));
    CKM(cudaMemsetAsync(m->d_status, 0, sizeof(int) * ST_COUNT, s));
    CKM(cudaMemcpyAsync(m->d_X, desc->X_ref, sizeof(double) * 3 * m->n_nodes, cudaMemcpyHostToDevice, s));
    {
        std::vector<Mat<float>> mf;
        std::vector<Mat<double>> md;
        for (auto &mm : m->h_mats) {
            mf.push_back(to_mat<float>(mm));
            md.push_back(to_mat<double>(mm));
        }
        CKM(cudaMemcpy(m->d_mats_f, mf.data(), sizeof(Mat<float>) * mf.size(), cudaMemcpyHostToDevice));
        CKM(cudaMemcpy(m->d_mats_d, md.data(), sizeof(Mat<double>) * md.size(), cudaMemcpyHostToDevice));
    }
    int base = 0;
    for (int bi = 0; bi < desc->n_blocks; ++bi) {
        st = build_block(m, desc, bi, base, s);
        if (st != TLFE_OK) return bail(st);
        base += desc->blocks[bi].n_elem;
        m->n_qp += (int64_t)desc->blocks[bi].n_elem * desc->blocks[bi].n_qp;
    }
    m->n_elem = base;
    st = build_fused_plan(m);
    if (st != TLFE_OK) return bail(st);
    if (m->scatter == TLFE_SCATTER_SORTED) {
        // transpose of the position -> node map: for each node its positions in
        // ascending order, which fixes the order of its sum
        const std::vector<int32_t> &pn = m->h_part_node;
        m->n_part = (int64_t)pn.size();
        std::vector<int64_t> ptr((size_t)m->n_nodes + 1, 0);
        for (int32_t n : pn)
            if (n >= 0) ptr[(size_t)n + 1]++;
        for (int n = 0; n < m->n_nodes; ++n) ptr[n + 1] += ptr[n];
        std::vector<int32_t> pos((size_t)std::max<int64_t>(1, ptr[m->n_nodes]));
        std::vector<int64_t> fill(ptr.begin(), ptr.end() - 1);
        for (int64_t k = 0; k < m->n_part; ++k)
            if (pn[k] >= 0) pos[fill[pn[k]]++] = (int32_t)k;
        const size_t rs = m->precision == TLFE_FP32 ? 4 : 8;
        m->d_part_ptr = (int64_t *)dalloc(m, sizeof(int64_t) * ptr.size(), &ae);
        m->d_part_pos = (int32_t *)dalloc(m, sizeof(int32_t) * pos.size(), &ae);
        m->d_part = dalloc(m, rs * 2 * 3 * (size_t)std::max<int64_t>(1, m->n_part), &ae);
        if (ae != cudaSuccess) return bail(cuda_fail(ae, "cudaMalloc (sorted scatter)"));
        CKM(cudaMemcpy(m->d_part_ptr, ptr.data(), sizeof(int64_t) * ptr.size(), cudaMemcpyHostToDevice));
        CKM(cudaMemcpy(m->d_part_pos, pos.data(), sizeof(int32_t) * pos.size(), cudaMemcpyHostToDevice));
        m->h_part_node.clear();
        m->h_part_node.shrink_to_fit();
    }
    int h_status[ST_COUNT];
    CKM(cudaMemcpy(h_status, m->d_status, sizeof(h_status), cudaMemcpyDeviceToHost));
    if (h_status[ST_INVERTED] > 0)
        return bail(fail(TLFE_E_INVERTED, std::to_string(h_status[ST_INVERTED]) +
                                              " element(s) with J_p <= 0 in the reference configuration"));
    CKM(cudaMemsetAsync(m->d_status, 0, sizeof(int) * ST_COUNT, s));
    CKM(cudaStreamSynchronize(s));
#undef CKM
    *out = m;
    return TLFE_OK;
}

extern "C" tlfe_status tlfe_destroy_mesh(tlfe_mesh *m)
{
    TLFE_TRACE("tlfe_destroy_mesh");
    if (!m) return TLFE_OK;
    cudaDeviceSynchronize();
    destroy_newton(m);
    destroy_graphs(m);
    destroy_host_stage(m);
    for (void *p : m->allocs) cudaFree(p);
    cudaFree(m->d_con_sh);
    cudaFree(m->d_con_gp);
    cudaFree(m->d_con_c);
    cudaFree(m->d_con_nd);
    cudaFree(m->d_con_bad);
    delete m->fused;
    delete m;
    return TLFE_OK;
}

extern "C" tlfe_status tlfe_get_mesh_info(const tlfe_mesh *m, tlfe_mesh_info *info)
{
    TLFE_TRACE("tlfe_get_mesh_info");
    if (!m || !info) return fail(TLFE_E_INVALID, "NULL argument");
    info->n_nodes = m->n_nodes;
    info->n_elem = m->n_elem;
    info->n_blocks = (int)m->blocks.size();
    info->precision = m->precision;
    info->scatter = m->scatter;
    info->n_qp = m->n_qp;
    int nc = 0;
    for (auto &B : m->blocks) nc = std::max(nc, B.n_colors);
    info->n_colors = m->scatter == TLFE_SCATTER_COLOR ? nc : 0;
    const int64_t rs = m->precision == TLFE_FP32 ? 4 : 8;
    int64_t eb = 0;  // element-side bytes: H, wJ, local indices, tile node lists, material arrays
    int naff = 0;
    for (auto &B : m->blocks) {
        if (B.use_affine) {
            eb += (int64_t)B.n_elem * AFF_ROWS * rs;              // J^{-1} and det J
            ++naff;
        } else {
            eb += (int64_t)B.n_elem * (B.nq * B.npe * 3 * rs + B.nq * rs);  // slab: h_i and w J_p
        }
        if (wpe_path(B.et, B.use_affine))   // warp per element: connectivity and slot element ids
            eb += (int64_t)B.n_elem * B.npe * 4 + (int64_t)B.n_tiles * TILE * 4;
        else
            eb += (int64_t)B.n_tiles * B.meta_bytes;                    // per-tile metadata records
        if (B.d_emat) eb += (int64_t)B.n_elem * 4;
        if (B.d_elam) eb += (int64_t)B.n_elem * 2 * rs;
    }
    const int64_t nb = (int64_t)m->n_nodes * 3 * rs;    // one node array in the mesh precision
    const int64_t nu = (int64_t)m->n_nodes * 3 * 8;     // the FP64 displacement
    bool visc = false;
    for (auto &B : m->blocks) visc = visc || B.visc;
    info->stream_bytes_force = eb + nu + nb * (visc ? 2 : 1);           // u (+udot) read, f written
    info->stream_bytes_matvec = eb + nu + nb * (visc ? 3 : 2);          // + v read
    info->stream_bytes_vjp = eb + nu + nb * (visc ? 4 : 2) + (int64_t)m->n_elem * 16;  // u, udot, r; g_u, g_udot; g_theta
    info->device_bytes = m->device_bytes;
    info->n_affine_blocks = naff;
    info->n_passes = 0;
    for (auto &B : m->blocks)
        if (B.n_elem > 0) info->n_passes += (int)B.color_tile_off.size() - 1;
    info->patch_layout = m->patch_layout;
    int64_t pl = 0, pp = 0;
    for (auto &B : m->blocks)
        if (!wpe_path(B.et, B.use_affine)) {
            pl += B.patch_loads;
            pp += B.patch_passes;
        }
    info->patch_passes = pl > 0 ? (double)pp / (double)pl : 1.0;
    info->n_fused_passes = m->fused ? (int)m->fused->passes.size() : 0;
    info->n_fused_items = m->fused ? m->fused->n_items : 0;
    // element-kernel launches of one force / operator-product call in the
    // current launch mode (the sorted scatter adds one node-sum kernel)
    for (int o = 0; o < 2; ++o) {
        const bool fused = m->fused && m->launch_mode != TLFE_LAUNCH_PER_PASS &&
                           (m->launch_mode == TLFE_LAUNCH_FUSED || m->fused->on[o]);
        int n = fused ? 1 : 0;
        for (size_t bi = 0; bi < m->blocks.size(); ++bi) {
            const BlockStore &B = m->blocks[bi];
            if (B.n_elem == 0 || (fused && m->fused->covered[bi])) continue;
            for (int c = 0; c + 1 < (int)B.color_tile_off.size(); ++c)
                if (B.color_tile_off[c + 1] > B.color_tile_off[c]) ++n;
        }
        if (m->scatter == TLFE_SCATTER_SORTED) ++n;
        (o == 0 ? info->launches_force : info->launches_matvec) = n;
    }
    info->force_matvec_fused = fm_eligible(m) ? 1 : 0;
    info->stream_bytes_force_matvec = eb + nu + nb * (visc ? 4 : 3);  // u (+udot), v read; f, y written
    return TLFE_OK;
}

extern "C" tlfe_status tlfe_get_colors(const tlfe_mesh *m, int32_t *colors)
{
    TLFE_TRACE("tlfe_get_colors");
    if (!m || !colors) return fail(TLFE_E_INVALID, "NULL argument");
    for (auto &B : m->blocks)
        for (int k = 0; k < B.n_elem; ++k) colors[B.elem_base + k] = B.colors.empty() ? -1 : B.colors[k];
    return TLFE_OK;
}

extern "C" tlfe_status tlfe_sync(tlfe_mesh *m, void *stream, int64_t *n_inverted)
{
    TLFE_TRACE("tlfe_sync");
    if (!m) return fail(TLFE_E_INVALID, "mesh is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    int h[ST_COUNT];
    CK(cudaMemcpyAsync(h, m->d_status, sizeof(h), cudaMemcpyDeviceToHost, s));
    CK(cudaMemsetAsync(m->d_status, 0, sizeof(h), s));
    CK(cudaStreamSynchronize(s));
    if (n_inverted) *n_inverted = h[ST_INVERTED];
    if (h[ST_TIMEOUT]) return fail(TLFE_E_TIMEOUT, "a bounded device wait ran out");
    if (h[ST_BOUNDS])
        return fail(TLFE_E_INVALID, std::to_string(h[ST_BOUNDS]) +
                                        " table index(es) out of range in the element kernels (bounds-checked build)");
    if (h[ST_NONFINITE]) return fail(TLFE_E_NONFINITE, "non-finite value met on the device");
    if (h[ST_INVERTED]) return fail(TLFE_E_INVERTED, std::to_string(h[ST_INVERTED]) + " quadrature point(s) with J <= 0");
    return TLFE_OK;
}

// ---------------------------------------------------------------------------
// element operations
// ---------------------------------------------------------------------------

namespace tlfe {

template <typename R> static const Mat<R> *mats_of(const tlfe_mesh *m);
template <> const Mat<float> *mats_of<float>(const tlfe_mesh *m) { return m->d_mats_f; }
template <> const Mat<double> *mats_of<double>(const tlfe_mesh *m) { return m->d_mats_d; }

// material mode of pass c of block B: the pass's law, with the viscous term
// when a velocity is given and an element of the pass is damped
static int pass_mat_mode(const BlockStore &B, int c, bool have_ud)
{
    const bool visc = have_ud && B.pass_visc[c];
    if (B.pass_model[c] == MODEL_NH) return visc ? MAT_NH_KV : MAT_NH;
    if (B.pass_model[c] == MODEL_SVK) return visc ? MAT_SVK_KV : MAT_SVK;
    return MAT_ANY;
}

// fill the block-independent fields of an element launch for block B
template <typename R> static void block_params(tlfe_mesh *m, const BlockStore &B, KParams<R> &p)
{
    p.umax = B.umax;
    p.tnode_off = B.d_toff;
    p.tnodes = B.d_tnodes;
    p.lidx = B.d_lidx;
    p.meta = B.d_meta;
    p.meta_bytes = B.meta_bytes;
    p.umaxp = B.meta_umaxp;
    p.eid = B.d_eid;
    p.conn = B.d_conn;
    p.elem_base = B.elem_base;
    p.slab = (const R *)B.d_slab;
    p.aff = B.use_affine ? (const R *)B.d_aff : nullptr;
    p.emat = B.d_emat;
    p.elam = (const R *)B.d_elam;
    p.evol = (const R *)B.d_evol;
    p.mats = B.d_emat ? mats_of<R>(m) : nullptr;
    p.mat0 = to_mat<R>(m->h_mats[B.uniform_body >= 0 ? B.uniform_body : 0]);
    p.status = m->d_status;
    p.part_base = B.part_base;
    p.n_nodes = m->n_nodes;
    p.n_elem_total = m->n_elem;
    p.n_mats = m->n_bodies;
    p.n_part = m->n_part;
    p.n_elem_block = B.n_elem;
}

// the launch schedule of (OP, block bi): from the cache, else from the occupancy API
template <int OP, typename R>
static tlfe_status block_sched(tlfe_mesh *m, int bi, int mat, LaunchSched *out)
{
    const BlockStore &B = m->blocks[bi];
    const auto key = std::make_tuple(OP, bi, mat, (int)sizeof(R));
    auto it = m->sched.find(key);
    if (it == m->sched.end()) {
        std::string why;
        LaunchSched ls;
        ls.wpb = 0;  // best CTA size
        ls.resident = occupancy_op<OP, R>(B.et, B.nq, B.use_affine, mat, B.umax, B.meta_bytes, &ls.wpb, &why);
        if (ls.resident <= 0) return fail(TLFE_E_UNSUPPORTED, "element kernel cannot be made resident: " + why);
        it = m->sched.emplace(key, ls).first;
    }
    *out = it->second;
    return TLFE_OK;
}

// launch one element kernel per pass of block bi, each with its material
// mode's schedule (or with `fixed`, for the passes of mode only_mat alone)
template <int OP, typename R>
static tlfe_status launch_block(tlfe_mesh *m, int bi, KParams<R> p, cudaStream_t s,
                                const LaunchSched *fixed = nullptr, int only_mat = -1)
{
    const BlockStore &B = m->blocks[bi];
    const int n_passes = (int)B.color_tile_off.size() - 1;
    for (int c = 0; c < n_passes; ++c) {
        p.tile_begin = B.color_tile_off[c];
        p.tile_end = B.color_tile_off[c + 1];
        const int tiles = p.tile_end - p.tile_begin;
        if (tiles <= 0) continue;
        p.visc = (B.pass_visc[c] && p.ud) ? 1 : 0;
        p.mat_mode = pass_mat_mode(B, c, p.ud != nullptr);
        if (only_mat >= 0 && p.mat_mode != only_mat) continue;
        LaunchSched ls;
        if (fixed) {
            ls = *fixed;
        } else {
            tlfe_status st = block_sched<OP, R>(m, bi, p.mat_mode, &ls);
            if (st != TLFE_OK) return st;
        }
        p.tile_chunk = ls.chunk;
        p.rmw_scatter = m->scatter == TLFE_SCATTER_COLOR ? 1 : 0;
        // one warp per tile (per element on the warp-per-element path) at a
        // time, persistent over the resident warps
        const int units = wpe_path(B.et, B.use_affine) ? tiles * TILE : tiles;
        const int warps = std::min(units, std::max(1, ls.resident / ls.wpb) * ls.wpb * m->n_sm);
        const int grid = std::max(1, (warps + ls.wpb - 1) / ls.wpb);
        cudaError_t e = launch_op<OP, R>(B.et, B.nq, p, grid, ls.wpb, s);
        if (e != cudaSuccess) return cuda_fail(e, "element kernel launch");
    }
    return TLFE_OK;
}

template <int OP, typename R>
static tlfe_status run_block_op(tlfe_mesh *m, int bi, KParams<R> p, cudaStream_t s)
{
    block_params<R>(m, m->blocks[bi], p);
    return launch_block<OP, R>(m, bi, p, s);
}

// sorted scatter, second half: out[n] = sum of node n's partials in ascending
// position order, for one or two output fields at once (part1 / out1 may be
// null). One thread per node: it reads the node's position range and
// positions once for both fields, loads up to four partial rows before it
// adds them, and adds in ascending position order, so the result repeats bit
// for bit; nodes in no element get 0.
template <typename R>
__global__ void k_node_sum(int64_t n_nodes, const int64_t *__restrict__ ptr, const int32_t *__restrict__ pos,
                           const R *__restrict__ part0, R *__restrict__ out0, const R *__restrict__ part1,
                           R *__restrict__ out1)
{
    for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < n_nodes;
         n += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k0 = ptr[n], k1 = ptr[n + 1];
        R a[3] = {R(0), R(0), R(0)}, b[3] = {R(0), R(0), R(0)};
        for (int64_t k = k0; k < k1; k += 4) {
            int64_t q[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) q[j] = k + j < k1 ? (int64_t)pos[k + j] * 3 : -1;
            R v[4][3], w[4][3];
#pragma unroll
            for (int j = 0; j < 4; ++j)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    v[j][c] = q[j] >= 0 ? part0[q[j] + c] : R(0);
                    w[j][c] = (part1 && q[j] >= 0) ? part1[q[j] + c] : R(0);
                }
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (q[j] >= 0)
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        a[c] += v[j][c];
                        b[c] += w[j][c];
                    }
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) out0[3 * n + c] = a[c];
        if (out1)
#pragma unroll
            for (int c = 0; c < 3; ++c) out1[3 * n + c] = b[c];
    }
}

// whether OP runs as the fused persistent launch on this mesh (launch mode,
// and the autotuner's choice in TLFE_LAUNCH_AUTO)
template <int OP, typename R> static bool use_fused(const tlfe_mesh *m)
{
    if constexpr (sizeof(R) != 4 || (OP != OP_FORCE && OP != OP_MATVEC)) {
        return false;
    } else {
        if (!m->fused || m->launch_mode == TLFE_LAUNCH_PER_PASS) return false;
        return m->launch_mode == TLFE_LAUNCH_FUSED || m->fused->on[OP == OP_FORCE ? 0 : 1];
    }
}

// the fused launch of OP over every covered pass: one parameter-table entry
// per pass (the call's fields of `base`, the block's layout, the pass's tile
// range and material mode), the item counter zeroed, all resident CTAs of the
// schedule (`fixed`, or the plan's: tuned, else from the occupancy API)
template <int OP>
static tlfe_status run_fused(tlfe_mesh *m, const KParams<float> &base, cudaStream_t s,
                             const LaunchSched *fixed = nullptr)
{
    FusedPlan &fp = *m->fused;
    const int o = OP == OP_FORCE ? 0 : 1;
    static thread_local FusedArgs<float> a;  // 17 KB: kept off the stack
    memset(&a, 0, sizeof(a));
    a.n_items = fp.n_items;
    a.items = fp.d_items;
    a.counter = fp.d_counter + o;
    a.wreg = (int)fp.wreg[o];
    for (size_t k = 0; k < fp.passes.size(); ++k) {
        const BlockStore &B = m->blocks[fp.passes[k].first];
        const int c = fp.passes[k].second;
        KParams<float> p = base;
        block_params<float>(m, B, p);
        p.tile_begin = B.color_tile_off[c];
        p.tile_end = B.color_tile_off[c + 1];
        p.visc = (B.pass_visc[c] && p.ud) ? 1 : 0;
        p.mat_mode = pass_mat_mode(B, c, p.ud != nullptr);
        p.tile_chunk = 0;
        p.rmw_scatter = 0;
        a.pass[k] = p;
        a.kind[k] = fused_code(B.et, B.nq) * MAT_N + p.mat_mode;
    }
    LaunchSched ls = fixed ? *fixed : fp.sched[o];
    if (ls.resident <= 0) {
        ls.wpb = 0;
        ls.resident = occupancy_fused<OP, float>(fp.wreg[o], &ls.wpb);
        if (ls.resident <= 0) return fail(TLFE_E_UNSUPPORTED, "fused element kernel cannot be made resident");
        if (!fixed) fp.sched[o] = ls;
    }
    const int warps = std::min(fp.n_items, std::max(1, ls.resident / ls.wpb) * ls.wpb * m->n_sm);
    const int grid = std::max(1, (warps + ls.wpb - 1) / ls.wpb);
    CK(cudaMemsetAsync(a.counter, 0, sizeof(int), s));
    cudaError_t e = launch_fused<OP, float>(a, grid, ls.wpb, s);
    if (e != cudaSuccess) return cuda_fail(e, "fused element kernel launch");
    return TLFE_OK;
}

template <int OP, typename R>
tlfe_status run_op(tlfe_mesh *m, const void *u, const void *ud, const void *v, void *out0, void *out1,
                   double *gth, double aM, double aK, double aC, int sym_only, cudaStream_t s)
{
    KParams<R> p;
    memset(&p, 0, sizeof(p));
    p.u = (const double *)u;
    p.ud = (const R *)ud;
    p.v = (const R *)v;
    p.out0 = (R *)out0;
    p.out1 = (R *)out1;
    p.gth = gth;
    p.aM = R(aM);
    p.aK = R(aK);
    p.aC = R(aC);
    p.sym_only = sym_only;
    p.mass_only = (OP == OP_MATVEC && aK == 0.0 && aC == 0.0) ? 1 : 0;
    const size_t nb = sizeof(R) * 3 * (size_t)m->n_nodes;
    const bool sorted = m->scatter == TLFE_SCATTER_SORTED;
    if (sorted) {
        if (sizeof(R) != (m->precision == TLFE_FP32 ? 4u : 8u))
            return fail(TLFE_E_UNSUPPORTED, "sorted scatter: operation precision differs from the mesh's");
        p.part0 = (R *)m->d_part;
        p.part1 = p.part0 + 3 * std::max<int64_t>(1, m->n_part);
    } else {
        if (out0) CK(cudaMemsetAsync(out0, 0, nb, s));
        if (out1) CK(cudaMemsetAsync(out1, 0, nb, s));
    }
    const bool fused = use_fused<OP, R>(m);
    if constexpr (sizeof(R) == 4 && (OP == OP_FORCE || OP == OP_MATVEC)) {
        if (fused) {
            tlfe_status st = run_fused<OP>(m, p, s);
            if (st != TLFE_OK) return st;
        }
    }
    for (int bi = 0; bi < (int)m->blocks.size(); ++bi) {
        if (m->blocks[bi].n_elem == 0 || (fused && m->fused->covered[bi])) continue;
        tlfe_status st = run_block_op<OP, R>(m, bi, p, s);
        if (st != TLFE_OK) return st;
    }
    if (sorted) {
        const int64_t nn = m->n_nodes;
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((nn + 255) / 256, (int64_t)m->n_sm * 16));
        R *o0 = (R *)out0, *o1 = (R *)out1;
        if (!o0) {  // a single field given as the second one
            o0 = o1;
            o1 = nullptr;
        }
        if (o0 && nn > 0) {
            const R *q0 = o0 == (R *)out0 ? p.part0 : p.part1;
            k_node_sum<R><<<grid, 256, 0, s>>>(nn, m->d_part_ptr, m->d_part_pos, q0, o0, o1 ? p.part1 : nullptr, o1);
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) return cuda_fail(e, "k_node_sum launch");
        }
    }
    return TLFE_OK;
}


// The fused force + operator-product pass (OP_FM) exists for the tile
// kernels of FP32 T4, T10 and H8 blocks (not for Q27, whose affine blocks run
// the warp-per-element kernels); it replaces the two per-pass launches where
// neither operation runs as the persistent launch.
static bool fm_kernels(const tlfe_mesh *m)
{
    if (m->precision != TLFE_FP32) return false;
    for (const BlockStore &B : m->blocks)
        if (B.n_elem > 0 && B.et == ET_Q27) return false;
    return true;
}

bool fm_eligible(const tlfe_mesh *m)
{
    return m->fm_on && fm_kernels(m) && !use_fused<OP_FORCE, float>(m) && !use_fused<OP_MATVEC, float>(m);
}

tlfe_status force_matvec_op(tlfe_mesh *m, const void *u, const void *ud, const void *v, double aM, double aK,
                            double aC, void *f, void *y, cudaStream_t s)
{
    if (fm_eligible(m)) return run_op<OP_FM, float>(m, u, ud, v, f, y, nullptr, aM, aK, aC, 0, s);
    tlfe_status st;
    if (m->precision == TLFE_FP32) {
        st = run_op<OP_FORCE, float>(m, u, ud, nullptr, f, nullptr, nullptr, 0, 1, 0, 0, s);
        return st != TLFE_OK ? st : run_op<OP_MATVEC, float>(m, u, ud, v, y, nullptr, nullptr, aM, aK, aC, 0, s);
    }
    st = run_op<OP_FORCE, double>(m, u, ud, nullptr, f, nullptr, nullptr, 0, 1, 0, 0, s);
    return st != TLFE_OK ? st : run_op<OP_MATVEC, double>(m, u, ud, v, y, nullptr, nullptr, aM, aK, aC, 0, s);
}

// ---------------------------------------------------------------------------
// Autotuner: time every resident CTA size (4, 2, 1 warps) and both tile
// assignments (interleaved, contiguous runs) of each block's force, operator
// and adjoint kernels on the caller's inputs, with outputs in scratch arrays,
// and keep the fastest per (op, block, material mode).
// ---------------------------------------------------------------------------

template <int OP, typename R>
static tlfe_status tune_block(tlfe_mesh *m, int bi, KParams<R> p, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1)
{
    const BlockStore &B = m->blocks[bi];
    block_params<R>(m, B, p);
    std::vector<int> modes;  // the material modes of the block's passes
    for (int c = 0; c + 1 < (int)B.color_tile_off.size(); ++c) {
        const int mat = pass_mat_mode(B, c, p.ud != nullptr);
        if (std::find(modes.begin(), modes.end(), mat) == modes.end()) modes.push_back(mat);
    }
    for (int mat : modes) {
        LaunchSched best;
        float best_ms = 1e30f;
        for (int wpb : {4, 2, 1}) {
            std::string why;
            LaunchSched ls;
            ls.wpb = wpb;
            ls.resident = occupancy_op<OP, R>(B.et, B.nq, B.use_affine, mat, B.umax, B.meta_bytes, &ls.wpb, &why);
            if (ls.resident <= 0) continue;
            for (int chunk : {0, 1}) {
                ls.chunk = chunk;
                tlfe_status st = launch_block<OP, R>(m, bi, p, s, &ls, mat);  // warm-up
                if (st != TLFE_OK) return st;
                float ms[3];
                for (int r = 0; r < 3; ++r) {
                    CK(cudaEventRecord(e0, s));
                    st = launch_block<OP, R>(m, bi, p, s, &ls, mat);
                    if (st != TLFE_OK) return st;
                    CK(cudaEventRecord(e1, s));
                    CK(cudaEventSynchronize(e1));
                    CK(cudaEventElapsedTime(&ms[r], e0, e1));
                }
                std::sort(ms, ms + 3);
                if (ms[1] < best_ms) {
                    best_ms = ms[1];
                    best = ls;
                }
            }
        }
        if (best.resident <= 0)
            return fail(TLFE_E_UNSUPPORTED, "no resident configuration for block " + std::to_string(bi));
        best.tuned = true;
        m->sched[std::make_tuple(OP, bi, mat, (int)sizeof(R))] = best;
    }
    return TLFE_OK;
}

// median of three timed runs of `launch` (after one untimed run), in ms
template <typename F>
static tlfe_status time_median3(F launch, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1, float *out)
{
    tlfe_status st = launch();
    if (st != TLFE_OK) return st;
    float ms[3];
    for (int r = 0; r < 3; ++r) {
        CK(cudaEventRecord(e0, s));
        st = launch();
        if (st != TLFE_OK) return st;
        CK(cudaEventRecord(e1, s));
        CK(cudaEventSynchronize(e1));
        CK(cudaEventElapsedTime(&ms[r], e0, e1));
    }
    std::sort(ms, ms + 3);
    *out = ms[1];
    return TLFE_OK;
}

// The fused launch of OP at every resident CTA size (4, 2, 1 warps) against
// the per-pass launches (with their tuned schedules) of the passes it covers;
// keeps the fastest schedule and, in TLFE_LAUNCH_AUTO, the faster mode.
template <int OP>
static tlfe_status tune_fused(tlfe_mesh *m, KParams<float> p, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1)
{
    FusedPlan &fp = *m->fused;
    const int o = OP == OP_FORCE ? 0 : 1;
    float per_pass = 0.f;
    tlfe_status st = time_median3(
        [&]() -> tlfe_status {
            for (int bi = 0; bi < (int)m->blocks.size(); ++bi) {
                if (!fp.covered[bi]) continue;
                tlfe_status s2 = run_block_op<OP, float>(m, bi, p, s);
                if (s2 != TLFE_OK) return s2;
            }
            return TLFE_OK;
        },
        s, e0, e1, &per_pass);
    if (st != TLFE_OK) return st;
    LaunchSched best;
    float best_ms = 1e30f;
    for (int wpb : {4, 2, 1}) {
        LaunchSched ls;
        ls.wpb = wpb;
        ls.resident = occupancy_fused<OP, float>(fp.wreg[o], &ls.wpb);
        if (ls.resident <= 0) continue;
        float ms = 0.f;
        st = time_median3([&]() { return run_fused<OP>(m, p, s, &ls); }, s, e0, e1, &ms);
        if (st != TLFE_OK) return st;
        if (ms < best_ms) {
            best_ms = ms;
            best = ls;
        }
    }
    if (best.resident <= 0) return TLFE_OK;  // keep the per-pass launches
    best.tuned = true;
    fp.sched[o] = best;
    fp.on[o] = best_ms <= per_pass;
    return TLFE_OK;
}

template <typename R>
static tlfe_status tune_all(tlfe_mesh *m, const double *u, const void *ud, const void *v, cudaStream_t s)
{
    const size_t nb = sizeof(R) * 3 * (size_t)m->n_nodes;
    void *o0 = nullptr, *o1 = nullptr;
    double *gth = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    tlfe_status st = TLFE_OK;
    cudaError_t e = cudaMalloc(&o0, nb);
    if (e == cudaSuccess) e = cudaMalloc(&o1, nb);
    if (e == cudaSuccess) e = cudaMalloc(&gth, sizeof(double) * 2 * std::max(1, m->n_elem));
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e != cudaSuccess) st = cuda_fail(e, "tlfe_autotune scratch");
    KParams<R> p;
    memset(&p, 0, sizeof(p));
    p.u = u;
    p.ud = (const R *)ud;
    p.v = (const R *)v;
    p.out0 = (R *)o0;
    p.out1 = (R *)o1;
    if (m->scatter == TLFE_SCATTER_SORTED && sizeof(R) == (m->precision == TLFE_FP32 ? 4u : 8u)) {
        p.part0 = (R *)m->d_part;   // time the kernels as they run: storing tile partials
        p.part1 = p.part0 + 3 * std::max<int64_t>(1, m->n_part);
    }
    p.gth = gth;
    p.aK = R(1);
    p.aC = R(1);
    for (int bi = 0; bi < (int)m->blocks.size() && st == TLFE_OK; ++bi) {
        if (m->blocks[bi].n_elem == 0) continue;
        st = tune_block<OP_FORCE, R>(m, bi, p, s, e0, e1);
        if (st == TLFE_OK && v) st = tune_block<OP_MATVEC, R>(m, bi, p, s, e0, e1);
        if (st == TLFE_OK && v) st = tune_block<OP_VJP, R>(m, bi, p, s, e0, e1);
    }
    if constexpr (sizeof(R) == 4) {
        if (st == TLFE_OK && m->fused) {
            st = tune_fused<OP_FORCE>(m, p, s, e0, e1);
            if (st == TLFE_OK && v) st = tune_fused<OP_MATVEC>(m, p, s, e0, e1);
        }
        // the fused force + operator-product pass: its own schedules, then one
        // fused pass against the two passes (with their tuned schedules) on
        // the caller's inputs; the faster is kept
        if (st == TLFE_OK && v && fm_kernels(m)) {
            m->fm_on = 1;
            for (int bi = 0; bi < (int)m->blocks.size() && st == TLFE_OK; ++bi)
                if (m->blocks[bi].n_elem > 0) st = tune_block<OP_FM, R>(m, bi, p, s, e0, e1);
            if (st == TLFE_OK && fm_eligible(m)) {
                float t_fm = 0.f, t_two = 0.f;
                st = time_median3([&]() { return run_op<OP_FM, float>(m, u, ud, v, o0, o1, nullptr, 0, 1, 1, 0, s); },
                                  s, e0, e1, &t_fm);
                if (st == TLFE_OK)
                    st = time_median3(
                        [&]() {
                            tlfe_status s2 = run_op<OP_FORCE, float>(m, u, ud, nullptr, o0, nullptr, nullptr, 0, 1, 0, 0, s);
                            return s2 != TLFE_OK ? s2
                                                 : run_op<OP_MATVEC, float>(m, u, ud, v, o1, nullptr, nullptr, 0, 1, 1, 0, s);
                        },
                        s, e0, e1, &t_two);
                if (st == TLFE_OK) m->fm_on = t_fm <= t_two ? 1 : 0;
            }
        }
    }
    cudaStreamSynchronize(s);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(o0);
    cudaFree(o1);
    cudaFree(gth);
    return st;
}

template tlfe_status run_op<OP_FORCE, float>(tlfe_mesh *, const void *, const void *, const void *, void *, void *, double *, double, double, double, int, cudaStream_t);
template tlfe_status run_op<OP_FORCE, double>(tlfe_mesh *, const void *, const void *, const void *, void *, void *, double *, double, double, double, int, cudaStream_t);
template tlfe_status run_op<OP_MATVEC, float>(tlfe_mesh *, const void *, const void *, const void *, void *, void *, double *, double, double, double, int, cudaStream_t);
template tlfe_status run_op<OP_MATVEC, double>(tlfe_mesh *, const void *, const void *, const void *, void *, void *, double *, double, double, double, int, cudaStream_t);
template tlfe_status run_op<OP_DIAG, float>(tlfe_mesh *, const void *, const void *, const void *, void *, void *, double *, double, double, double, int, cudaStream_t);
template tlfe_status run_op<OP_DIAG, double>(tlfe_mesh *, const void *, const void *, const void *, void *, void *, double *, double, double, double, int, cudaStream_t);
template tlfe_status run_op<OP_VJP, float>(tlfe_mesh *, const void *, const void *, const void *, void *, void *, double *, double, double, double, int, cudaStream_t);
template tlfe_status run_op<OP_VJP, double>(tlfe_mesh *, const void *, const void *, const void *, void *, void *, double *, double, double, double, int, cudaStream_t);
template tlfe_status run_op<OP_FM, float>(tlfe_mesh *, const void *, const void *, const void *, void *, void *, double *, double, double, double, int, cudaStream_t);

}  // namespace tlfe

static tlfe_status check_mesh_args(tlfe_mesh *m, std::initializer_list<const void *> req)
{
    if (!m) return fail(TLFE_E_INVALID, "mesh is NULL");
    for (const void *p : req)
        if (!p) return fail(TLFE_E_INVALID, "required array pointer is NULL");
    return TLFE_OK;
}

static bool all_affine(const tlfe_mesh *m)
{
    for (auto &B : m->blocks)
        if (B.n_elem > 0 && !B.affine) return false;
    return true;
}

tlfe_status tlfe::check_force_matvec(tlfe_mesh *m, const void *u, const void *v, const void *f, const void *y,
                                     double aM, double aK, double aC)
{
    tlfe_status st = check_mesh_args(m, {u, v, f, y});
    if (st != TLFE_OK) return st;
    if (f == y) return fail(TLFE_E_INVALID, "f and y must be different arrays");
    if (!std::isfinite(aM) || !std::isfinite(aK) || !std::isfinite(aC)) return fail(TLFE_E_INVALID, "non-finite coefficient");
    if (aM != 0.0 && !all_affine(m)) return fail(TLFE_E_UNSUPPORTED, "consistent mass needs affine elements");
    return TLFE_OK;
}

extern "C" tlfe_status tlfe_internal_force(tlfe_mesh *m, const void *u, const void *ud, void *f, void *stream)
{
    TLFE_TRACE("tlfe_internal_force");
    tlfe_status st = check_mesh_args(m, {u, f});
    if (st != TLFE_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    return m->precision == TLFE_FP32
               ? run_op<OP_FORCE, float>(m, u, ud, nullptr, f, nullptr, nullptr, 0, 1, 0, 0, s)
               : run_op<OP_FORCE, double>(m, u, ud, nullptr, f, nullptr, nullptr, 0, 1, 0, 0, s);
}

extern "C" tlfe_status tlfe_internal_force_host(tlfe_mesh *m, const void *u_h, const void *ud_h, void *f_h,
                                                void *stream)
{
    TLFE_TRACE("tlfe_internal_force_host");
    tlfe_status st = check_mesh_args(m, {u_h, f_h});
    if (st != TLFE_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t nb = (size_t)3 * m->n_nodes * (m->precision == TLFE_FP32 ? 4 : 8);
    const size_t nu = (size_t)3 * m->n_nodes * 8;  // the displacement is FP64 in both precisions
    if (!m->d_stage) CKA(m->d_stage, nu + 2 * nb, m);
    char *du = (char *)m->d_stage, *dud = du + nu, *df = dud + nb;
    CK(cudaMemcpyAsync(du, u_h, nu, cudaMemcpyHostToDevice, s));
    if (ud_h) CK(cudaMemcpyAsync(dud, ud_h, nb, cudaMemcpyHostToDevice, s));
    st = tlfe_internal_force(m, du, ud_h ? dud : nullptr, df, stream);
    if (st != TLFE_OK) return st;
    CK(cudaMemcpyAsync(f_h, df, nb, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return TLFE_OK;
}

extern "C" tlfe_status tlfe_tangent_matvec(tlfe_mesh *m, const void *u, const void *ud, const void *v, double aM,
                                           double aK, double aC, void *y, void *stream)
{
    TLFE_TRACE("tlfe_tangent_matvec");
    tlfe_status st = check_mesh_args(m, {u, v, y});
    if (st != TLFE_OK) return st;
    if (!std::isfinite(aM) || !std::isfinite(aK) || !std::isfinite(aC)) return fail(TLFE_E_INVALID, "non-finite coefficient");
    if (aM != 0.0 && !all_affine(m)) return fail(TLFE_E_UNSUPPORTED, "consistent mass needs affine elements");
    cudaStream_t s = (cudaStream_t)stream;
    return m->precision == TLFE_FP32
               ? run_op<OP_MATVEC, float>(m, u, ud, v, y, nullptr, nullptr, aM, aK, aC, 0, s)
               : run_op<OP_MATVEC, double>(m, u, ud, v, y, nullptr, nullptr, aM, aK, aC, 0, s);
}

extern "C" tlfe_status tlfe_newton_operator(tlfe_mesh *m, const void *u, const void *ud, const void *v, double aM,
                                            double aK, double aC, void *y, void *stream)
{
    TLFE_TRACE("tlfe_newton_operator");
    tlfe_status st = check_mesh_args(m, {u, v, y});
    if (st != TLFE_OK) return st;
    if (!std::isfinite(aM) || !std::isfinite(aK) || !std::isfinite(aC)) return fail(TLFE_E_INVALID, "non-finite coefficient");
    if (aM != 0.0 && !all_affine(m)) return fail(TLFE_E_UNSUPPORTED, "consistent mass needs affine elements");
    cudaStream_t s = (cudaStream_t)stream;
    return m->precision == TLFE_FP32
               ? run_op<OP_MATVEC, float>(m, u, ud, v, y, nullptr, nullptr, aM, aK, aC, 1, s)
               : run_op<OP_MATVEC, double>(m, u, ud, v, y, nullptr, nullptr, aM, aK, aC, 1, s);
}

extern "C" tlfe_status tlfe_jacobi_diag(tlfe_mesh *m, const void *u, const void *ud, double aM, double aK, double aC,
                                        void *d, void *stream)
{
    TLFE_TRACE("tlfe_jacobi_diag");
    tlfe_status st = check_mesh_args(m, {u, d});
    if (st != TLFE_OK) return st;
    if (aM != 0.0 && !all_affine(m)) return fail(TLFE_E_UNSUPPORTED, "consistent mass needs affine elements");
    cudaStream_t s = (cudaStream_t)stream;
    return m->precision == TLFE_FP32
               ? run_op<OP_DIAG, float>(m, u, ud, nullptr, d, nullptr, nullptr, aM, aK, aC, 1, s)
               : run_op<OP_DIAG, double>(m, u, ud, nullptr, d, nullptr, nullptr, aM, aK, aC, 1, s);
}

extern "C" tlfe_status tlfe_vjp(tlfe_mesh *m, const void *u, const void *ud, const void *cot, void *g_u, void *g_ud,
                                double *g_th, void *stream)
{
    TLFE_TRACE("tlfe_vjp");
    tlfe_status st = check_mesh_args(m, {u, cot});
    if (st != TLFE_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t nb = (size_t)3 * m->n_nodes * (m->precision == TLFE_FP32 ? 4 : 8);
    if ((!g_u || !g_ud) && !m->d_scratch_vjp) CKA(m->d_scratch_vjp, 2 * nb, m);
    void *o0 = g_u ? g_u : m->d_scratch_vjp;
    void *o1 = g_ud ? g_ud : (char *)m->d_scratch_vjp + nb;
    return m->precision == TLFE_FP32
               ? run_op<OP_VJP, float>(m, u, ud, cot, o0, o1, g_th, 0, 1, 0, 0, s)
               : run_op<OP_VJP, double>(m, u, ud, cot, o0, o1, g_th, 0, 1, 0, 0, s);
}

extern "C" tlfe_status tlfe_autotune(tlfe_mesh *m, const double *u, const void *ud, const void *v, void *stream)
{
    TLFE_TRACE("tlfe_autotune");
    tlfe_status st = check_mesh_args(m, {u});
    if (st != TLFE_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    ++m->sched_gen;
    return m->precision == TLFE_FP32 ? tune_all<float>(m, u, ud, v, s) : tune_all<double>(m, u, ud, v, s);
}

extern "C" tlfe_status tlfe_set_launch_mode(tlfe_mesh *m, int32_t mode)
{
    TLFE_TRACE("tlfe_set_launch_mode");
    if (!m) return fail(TLFE_E_INVALID, "mesh is NULL");
    if (mode != TLFE_LAUNCH_AUTO && mode != TLFE_LAUNCH_PER_PASS && mode != TLFE_LAUNCH_FUSED)
        return fail(TLFE_E_INVALID, "bad launch mode");
    m->launch_mode = mode;
    ++m->sched_gen;
    return TLFE_OK;
}

extern "C" tlfe_status tlfe_set_elem_mu_lambda(tlfe_mesh *m, const double *mu_lambda_dev, void *stream)
{
    TLFE_TRACE("tlfe_set_elem_mu_lambda");
    tlfe_status st = check_mesh_args(m, {mu_lambda_dev});
    if (st != TLFE_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t rs = m->precision == TLFE_FP32 ? 4 : 8;
    for (auto &B : m->blocks) {
        if (B.n_tiles == 0) continue;
        if (!B.d_elam) {
            CKA(B.d_elam, rs * (size_t)B.n_tiles * TILE * 2, m);
            ++m->sched_gen;  // the blocks' launch parameters now carry the per-element array
        }
        cudaError_t e = launch_set_elam(m->precision, B.n_tiles, B.d_eid, mu_lambda_dev, B.d_elam, s);
        if (e != cudaSuccess) return cuda_fail(e, "tlfe_set_elem_mu_lambda");
    }
    // keep the FP64 twin used by the Newton step consistent
    if (tlfe_mesh *tw = newton_twin(m)) return tlfe_set_elem_mu_lambda(tw, mu_lambda_dev, stream);
    return TLFE_OK;
}

extern "C" const char *tlfe_last_error(void) { return tlfe::g_err.c_str(); }

extern "C" const char *tlfe_version(void) { return "tlfe 0.1 (sm_103a)"; }
