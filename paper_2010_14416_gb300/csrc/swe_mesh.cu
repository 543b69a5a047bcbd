// swe_mesh.cu -- host preprocessing (host code only; built by nvcc so it can
// share the device-side constants) of a triangular mesh for the fused step
// kernel: validation, counter-clockwise orientation, neighbours across shared
// edges (Section 4.2: the cells that share an edge with a cell), geometry of
// Eq 9 (|Omega_i|, L_ij n_ij) and Eq 15 (inscribed radius), a locality
// ordering of the cells, and the canonical orientation of every interior edge.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>

#include "swe_internal.h"

namespace swe {

namespace {

// Hilbert index of (x, y) on a 2^order x 2^order grid (the classic
// rotate-and-reflect recursion of the Hilbert curve, unrolled).
uint64_t hilbert_index(uint32_t x, uint32_t y, int order) {
    const uint32_t mask = (order >= 32) ? 0xFFFFFFFFu : ((1u << order) - 1u);
    uint64_t d = 0;
    for (uint32_t s = 1u << (order - 1); s > 0; s >>= 1) {
        const uint32_t rx = (x & s) ? 1u : 0u;
        const uint32_t ry = (y & s) ? 1u : 0u;
        d += (uint64_t)s * (uint64_t)s * ((3u * rx) ^ ry);
        // turn the quadrant into the canonical orientation; only the bits
        // below s are looked at afterwards
        if (ry == 0) {
            if (rx == 1) {
                x = mask - x;
                y = mask - y;
            }
            std::swap(x, y);
        }
    }
    return d;
}

// LSD radix sort of (key, index) pairs on the low `bits` bits of the key.
void radix_sort_pairs(std::vector<uint64_t>& key, std::vector<int64_t>& idx, int bits) {
    const size_t n = key.size();
    std::vector<uint64_t> k2(n);
    std::vector<int64_t> i2(n);
    for (int shift = 0; shift < bits; shift += 11) {
        size_t count[2049] = {0};
        for (size_t p = 0; p < n; ++p) ++count[((key[p] >> shift) & 2047u) + 1];
        for (int b = 0; b < 2048; ++b) count[b + 1] += count[b];
        for (size_t p = 0; p < n; ++p) {
            const size_t q = count[(key[p] >> shift) & 2047u]++;
            k2[q] = key[p];
            i2[q] = idx[p];
        }
        key.swap(k2);
        idx.swap(i2);
    }
}

}  // namespace

std::vector<int64_t> order_hilbert(const std::vector<double>& cx, const std::vector<double>& cy) {
    const int64_t n = (int64_t)cx.size();
    double x0 = cx[0], x1 = cx[0], y0 = cy[0], y1 = cy[0];
    for (int64_t i = 1; i < n; ++i) {
        x0 = std::min(x0, cx[i]); x1 = std::max(x1, cx[i]);
        y0 = std::min(y0, cy[i]); y1 = std::max(y1, cy[i]);
    }
    const int order = 20;
    const double span = std::max(std::max(x1 - x0, y1 - y0), 1e-300);
    const double scale = (double)((1u << order) - 1) / span;
    std::vector<uint64_t> key(n);
    std::vector<int64_t> idx(n);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        const uint32_t gx = (uint32_t)std::lround((cx[i] - x0) * scale);
        const uint32_t gy = (uint32_t)std::lround((cy[i] - y0) * scale);
        key[i] = hilbert_index(gx, gy, order);
        idx[i] = i;
    }
    radix_sort_pairs(key, idx, 2 * order);
    return idx;
}

std::vector<int64_t> order_rcm(int64_t n, const std::vector<int64_t>& nbr) {
    auto degree = [&](int64_t c) {
        int d = 0;
        for (int j = 0; j < 3; ++j) d += nbr[3 * c + j] >= 0;
        return d;
    };
    std::vector<int64_t> order;
    order.reserve(n);
    std::vector<int64_t> level(n, -1);
    std::vector<char> placed(n, 0);
    std::vector<int64_t> queue;
    queue.reserve(n);
    // BFS from `start` over unplaced cells; returns the last cell reached
    auto bfs_far = [&](int64_t start, std::vector<int64_t>& seen_list) {
        seen_list.clear();
        seen_list.push_back(start);
        level[start] = 0;
        size_t h = 0;
        int64_t last = start;
        while (h < seen_list.size()) {
            const int64_t c = seen_list[h++];
            last = c;
            for (int j = 0; j < 3; ++j) {
                const int64_t k = nbr[3 * c + j];
                if (k >= 0 && !placed[k] && level[k] < 0) {
                    level[k] = level[c] + 1;
                    seen_list.push_back(k);
                }
            }
        }
        for (int64_t c : seen_list) level[c] = -1;
        return last;
    };
    std::vector<int64_t> comp;
    for (int64_t seed = 0; seed < n; ++seed) {
        if (placed[seed]) continue;
        // pseudo-peripheral start: two sweeps to the far end of the component
        int64_t s = bfs_far(seed, comp);
        s = bfs_far(s, comp);
        // Cuthill-McKee ordering: BFS visiting neighbours by increasing degree
        const size_t base = order.size();
        order.push_back(s);
        placed[s] = 1;
        for (size_t h = base; h < order.size(); ++h) {
            const int64_t c = order[h];
            int64_t ks[3];
            int cnt = 0;
            for (int j = 0; j < 3; ++j) {
                const int64_t k = nbr[3 * c + j];
                if (k >= 0 && !placed[k]) ks[cnt++] = k;
            }
            std::sort(ks, ks + cnt, [&](int64_t p, int64_t q) {
                const int dp = degree(p), dq = degree(q);
                return dp != dq ? dp < dq : p < q;
            });
            for (int t = 0; t < cnt; ++t) {
                placed[ks[t]] = 1;
                order.push_back(ks[t]);
            }
        }
        std::reverse(order.begin() + base, order.end());
    }
    return order;
}

void match_cells(const std::vector<int64_t>& along, const std::vector<int64_t>& nbr, const std::vector<int32_t>& t,
                 std::vector<int64_t>& mate, std::vector<int>& rot) {
    const int64_t n = (int64_t)along.size();
    constexpr int64_t kWindow = 256;   // a partner comes at most this many places later
    std::vector<int64_t> pos(n);
    for (int64_t p = 0; p < n; ++p) pos[along[p]] = p;
    mate.assign(n, -1);
    rot.assign(n, 0);
    for (int64_t p = 0; p < n; ++p) {
        const int64_t c = along[p];
        if (mate[c] >= 0) continue;
        int64_t best = -1;
        int jc = 0;
        for (int j = 0; j < 3; ++j) {
            const int64_t k = nbr[3 * c + j];
            if (k < 0 || mate[k] >= 0 || pos[k] <= p || pos[k] > p + kWindow) continue;
            if (best < 0 || pos[k] < pos[best]) { best = k; jc = j; }
        }
        if (best < 0) continue;
        // the same edge in the partner, traversed the other way (both counter-clockwise)
        const int32_t a = t[3 * c + jc], b = t[3 * c + (jc + 1) % 3];
        int jk = -1;
        for (int j = 0; j < 3; ++j)
            if (t[3 * best + j] == b && t[3 * best + (j + 1) % 3] == a) jk = j;
        if (jk < 0) continue;
        mate[c] = best;
        mate[best] = c;
        rot[c] = jc;
        rot[best] = jk;
    }
}

std::vector<int64_t> place_pairs(const std::vector<int64_t>& order, const std::vector<int64_t>& mate) {
    const int64_t n = (int64_t)order.size();
    constexpr size_t kSegment = 64;    // cells per segment of only pairs or only unmatched cells
    std::vector<char> placed(n, 0);
    std::vector<int64_t> out;
    out.reserve(n);
    std::vector<int64_t> single;
    size_t taken = 0;
    for (int64_t p = 0; p < n; ++p) {
        const int64_t c = order[p];
        if (placed[c]) continue;
        if (mate[c] >= 0) {
            out.push_back(c);
            out.push_back(mate[c]);
            placed[c] = placed[mate[c]] = 1;
        } else {
            single.push_back(c);
            placed[c] = 1;
        }
        if (out.size() % kSegment == 0 && single.size() - taken >= kSegment) {
            out.insert(out.end(), single.begin() + taken, single.begin() + taken + kSegment);
            taken += kSegment;
        }
    }
    out.insert(out.end(), single.begin() + taken, single.end());
    return out;
}

int build_host_mesh(const double* nodes, int64_t n_nodes, const int32_t* tris, int64_t n,
                    const double* bathy, const double* manning, int reorder, bool pair_cells, HostMesh& M,
                    std::string& err) {
    if (!nodes || !tris || !bathy || !manning || n_nodes < 3 || n < 1) {
        err = "swe_mesh_create: null array or empty mesh";
        return SWE_EINVAL;
    }
    if (n >= (int64_t)kNbrMask || n_nodes >= ((int64_t)1 << 31)) {
        err = "swe_mesh_create: too many cells or nodes";
        return SWE_EINVAL;
    }
    M.n_cells = n;
    M.n_nodes = n_nodes;
    // orientation and validation, caller order
    std::vector<int32_t> t(3 * n);
    std::vector<double> cx(n), cy(n);
    int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad)
    for (int64_t i = 0; i < n; ++i) {
        int32_t v0 = tris[3 * i], v1 = tris[3 * i + 1], v2 = tris[3 * i + 2];
        if (v0 < 0 || v1 < 0 || v2 < 0 || v0 >= n_nodes || v1 >= n_nodes || v2 >= n_nodes ||
            v0 == v1 || v1 == v2 || v0 == v2) {
            bad |= 1;
            continue;
        }
        const double ax = nodes[2 * v0], ay = nodes[2 * v0 + 1];
        const double bx = nodes[2 * v1], by = nodes[2 * v1 + 1];
        const double qx = nodes[2 * v2], qy = nodes[2 * v2 + 1];
        const double a2 = (bx - ax) * (qy - ay) - (qx - ax) * (by - ay);
        if (!(a2 != 0.0) || !std::isfinite(a2)) { bad |= 2; continue; }
        if (!(manning[i] >= 0.0) || !std::isfinite(manning[i]) || !std::isfinite(bathy[i])) { bad |= 4; continue; }
        if (a2 < 0.0) std::swap(v1, v2);
        t[3 * i] = v0; t[3 * i + 1] = v1; t[3 * i + 2] = v2;
        cx[i] = (ax + bx + qx) / 3.0;
        cy[i] = (ay + by + qy) / 3.0;
    }
    if (bad & 1) { err = "swe_mesh_create: triangle with an out-of-range or repeated node"; return SWE_EMESH; }
    if (bad & 2) { err = "swe_mesh_create: triangle with zero or non-finite area"; return SWE_EMESH; }
    if (bad & 4) { err = "swe_mesh_create: negative or non-finite Manning coefficient, or non-finite bed"; return SWE_EINVAL; }

    // neighbours: bucket half-edges by their lower node, match within buckets
    std::vector<int64_t> start(n_nodes + 1, 0);
    for (int64_t s = 0; s < 3 * n; ++s) {
        const int32_t a = t[s], b = t[(s / 3) * 3 + (s % 3 + 1) % 3];
        ++start[std::min(a, b) + 1];
    }
    for (int64_t v = 0; v < n_nodes; ++v) start[v + 1] += start[v];
    std::vector<int64_t> fill(start.begin(), start.end() - 1);
    std::vector<int64_t> bucket(3 * n);
    for (int64_t s = 0; s < 3 * n; ++s) {
        const int32_t a = t[s], b = t[(s / 3) * 3 + (s % 3 + 1) % 3];
        bucket[fill[std::min(a, b)]++] = s;
    }
    std::vector<int64_t> nbr_old(3 * n, -1);
    int mesh_bad = 0;
#pragma omp parallel for schedule(dynamic, 4096) reduction(| : mesh_bad)
    for (int64_t v = 0; v < n_nodes; ++v) {
        const int64_t b0 = start[v], b1 = start[v + 1];
        auto other = [&](int64_t s) {
            const int32_t a = t[s], b = t[(s / 3) * 3 + (s % 3 + 1) % 3];
            return std::max(a, b);
        };
        // small buckets: sort by the upper node
        std::sort(bucket.begin() + b0, bucket.begin() + b1,
                  [&](int64_t p, int64_t q) { return other(p) != other(q) ? other(p) < other(q) : p < q; });
        int64_t p = b0;
        while (p < b1) {
            int64_t q = p + 1;
            while (q < b1 && other(bucket[q]) == other(bucket[p])) ++q;
            if (q - p > 2) { mesh_bad |= 1; p = q; continue; }
            if (q - p == 2) {
                const int64_t s0 = bucket[p], s1 = bucket[p + 1];
                if (s0 / 3 == s1 / 3) { mesh_bad |= 1; p = q; continue; }
                nbr_old[s0] = s1 / 3;
                nbr_old[s1] = s0 / 3;
            }
            p = q;
        }
    }
    if (mesh_bad) { err = "swe_mesh_create: an edge is shared by more than two triangles"; return SWE_EMESH; }

    // locality order
    std::vector<int64_t> order;
    if (reorder == SWE_REORDER_HILBERT) {
        order = order_hilbert(cx, cy);
    } else if (reorder == SWE_REORDER_RCM) {
        order = order_rcm(n, nbr_old);
    } else if (reorder == SWE_REORDER_NONE) {
        order.resize(n);
        std::iota(order.begin(), order.end(), 0);
    } else {
        err = "swe_mesh_create: unknown reorder mode";
        return SWE_EINVAL;
    }
    // FP32 meshes: pairs of adjacent cells, matched along the Hilbert order
    // whatever the mode, with their shared edge as local edge 0 of both: every
    // mode numbers each cell's edges alike (so sums them in the same order);
    // the RCM and Hilbert orders then place the pairs at (2p, 2p+1).  FP64
    // meshes (no pair kernel) keep the caller's local edge numbering.
    std::vector<int64_t> mate(n, -1);
    std::vector<int> rot(n, 0);
    if (pair_cells) {
        match_cells(reorder == SWE_REORDER_HILBERT ? order : order_hilbert(cx, cy), nbr_old, t, mate, rot);
        if (reorder != SWE_REORDER_NONE) order = place_pairs(order, mate);
    }
    M.perm = order;
    M.inv.assign(n, 0);
    for (int64_t c = 0; c < n; ++c) M.inv[order[c]] = c;

    M.tri.resize(3 * n);
    M.ln.resize(6 * n);
    M.inv_area.resize(n);
    M.rin.resize(n);
    M.z.resize(n);
    M.m.resize(n);
    M.code.resize(3 * n);
    M.len.resize(3 * n);
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < n; ++c) {
        const int64_t o = order[c];
        double perim = 0.0;
        for (int j = 0; j < 3; ++j) {
            const int jo = (j + rot[o]) % 3;   // local edge j is the caller's edge jo
            const int32_t a = t[3 * o + jo], b = t[3 * o + (jo + 1) % 3];
            M.tri[3 * c + j] = a;
            const double dx = nodes[2 * b] - nodes[2 * a];
            const double dy = nodes[2 * b + 1] - nodes[2 * a + 1];
            // outward normal of a counter-clockwise triangle, times the length
            M.ln[6 * c + 2 * j] = dy;
            M.ln[6 * c + 2 * j + 1] = -dx;
            M.len[3 * c + j] = std::sqrt(dx * dx + dy * dy);
            const int64_t k = nbr_old[3 * o + jo];
            if (k >= 0) {
                int32_t code = (int32_t)M.inv[k];
                if (k < o) code |= kFlipBit;  // the neighbour is the edge's left state
                M.code[3 * c + j] = code;
            } else {
                M.code[3 * c + j] = -1;  // boundary group 0: wall
            }
        }
        const int32_t v0 = t[3 * o], v1 = t[3 * o + 1], v2 = t[3 * o + 2];
        const double a2 = (nodes[2 * v1] - nodes[2 * v0]) * (nodes[2 * v2 + 1] - nodes[2 * v0 + 1]) -
                          (nodes[2 * v2] - nodes[2 * v0]) * (nodes[2 * v1 + 1] - nodes[2 * v0 + 1]);
        const double area = 0.5 * a2;
        // the perimeter summed in the caller's edge order, whatever the rotation
        for (int j = 0; j < 3; ++j) perim += M.len[3 * c + (j + 3 - rot[o]) % 3];
        M.inv_area[c] = 1.0 / area;
        M.rin[c] = 2.0 * area / perim;
        M.z[c] = bathy[o];
        M.m[c] = manning[o];
    }
    // boundary half-edges, sorted by node-pair key for swe_set_bc lookups
    std::vector<uint64_t> key;
    std::vector<int64_t> slot;
    for (int64_t s = 0; s < 3 * n; ++s) {
        if (M.code[s] >= 0) continue;
        const int32_t a = M.tri[s], b = M.tri[(s / 3) * 3 + (s % 3 + 1) % 3];
        key.push_back(((uint64_t)std::min(a, b) << 32) | (uint64_t)std::max(a, b));
        slot.push_back(s);
    }
    std::vector<int64_t> idx(key.size());
    std::iota(idx.begin(), idx.end(), 0);
    std::sort(idx.begin(), idx.end(), [&](int64_t p, int64_t q) { return key[p] < key[q]; });
    M.bkey.resize(key.size());
    M.bslot.resize(key.size());
    for (size_t r = 0; r < idx.size(); ++r) {
        M.bkey[r] = key[idx[r]];
        M.bslot[r] = slot[idx[r]];
    }
    return SWE_OK;
}

}  // namespace swe
