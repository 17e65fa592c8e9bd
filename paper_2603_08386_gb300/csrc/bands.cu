// ddhf_merge_bands: the boxes of a sensor processed as row bands (Sec. 3.5
// "Segmentation mask processing" and Eq. 12), computed on the host from what
// each band's context produced: its components in sensor coordinates and the
// labels of its first and last rows.
//
// Components that touch across a band boundary (8-connectivity between the
// last row of band b and the first row of band b + 1) are joined with a
// union-find; the joined component's box is the union of its parts' boxes
// and its pixel count their sum. From there the steps and their arithmetic
// match ddhf_boxes on a whole sensor: boxes with area < A_min are removed,
// Eq. 12 is tested in FP64 on every pair (each product rounded on its own),
// each round replaces every group of transitively close boxes by its union
// box, rounds repeat until no pair is close, and the result is sorted by
// (y0, x0, y1, x1, n_px). The grouping of a round does not depend on the order
// of the boxes, so neither does the result.
#include <stdint.h>

#include <algorithm>
#include <numeric>
#include <vector>

#include "ddhf.h"

namespace {

struct Box5 {
  int32_t x0, y0, x1, y1, n;
};

struct UnionFind {
  std::vector<int64_t> par;
  explicit UnionFind(int64_t n) : par((size_t)n) { std::iota(par.begin(), par.end(), 0); }
  int64_t find(int64_t x) {
    while (par[(size_t)x] != x) {
      par[(size_t)x] = par[(size_t)par[(size_t)x]];
      x = par[(size_t)x];
    }
    return x;
  }
  void unite(int64_t a, int64_t b) {
    a = find(a);
    b = find(b);
    if (a == b) return;
    if (a < b) std::swap(a, b);
    par[(size_t)a] = b;  // the smaller index becomes the root
  }
};

bool eq12_close(const Box5 &a, const Box5 &b, double alpha) {
  const int64_t dx2 = (int64_t)(a.x0 + a.x1) - (int64_t)(b.x0 + b.x1);
  const int64_t dy2 = (int64_t)(a.y0 + a.y1) - (int64_t)(b.y0 + b.y1);
  int64_t m = a.x1 - a.x0 + 1;
  m = std::max(m, (int64_t)(a.y1 - a.y0 + 1));
  m = std::max(m, (int64_t)(b.x1 - b.x0 + 1));
  m = std::max(m, (int64_t)(b.y1 - b.y0 + 1));
  const double lhs = (double)(dx2 * dx2 + dy2 * dy2);
  const double s = (2.0 * alpha) * (double)m;  // products only: each rounded on its own
  return lhs < s * s;
}

// Replace each group of boxes by its union box; groups from the union-find.
std::vector<Box5> union_groups(const std::vector<Box5> &in, UnionFind &uf) {
  std::vector<Box5> out;
  std::vector<int64_t> slot(in.size(), -1);
  for (size_t i = 0; i < in.size(); ++i) {
    const int64_t r = uf.find((int64_t)i);
    if (slot[(size_t)r] < 0) {
      slot[(size_t)r] = (int64_t)out.size();
      out.push_back(Box5{in[(size_t)r].x0, in[(size_t)r].y0, in[(size_t)r].x1,
                         in[(size_t)r].y1, 0});
    }
    Box5 &o = out[(size_t)slot[(size_t)r]];
    o.x0 = std::min(o.x0, in[i].x0);
    o.y0 = std::min(o.y0, in[i].y0);
    o.x1 = std::max(o.x1, in[i].x1);
    o.y1 = std::max(o.y1, in[i].y1);
    o.n += in[i].n;
  }
  return out;
}

}  // namespace

extern "C" ddhf_status ddhf_merge_bands(int32_t W, int32_t H, int32_t n_bands,
                                        const int32_t *band_row0, const int32_t *edge_labels,
                                        const ddhf_component *comps, const int64_t *comp_off,
                                        const ddhf_params *params, ddhf_box *boxes, int32_t cap,
                                        int32_t *n_boxes) {
  if (W < 1 || H < 1 || n_bands < 1 || !band_row0 || !edge_labels || !comp_off || !params ||
      !n_boxes || cap < 0 || (cap > 0 && !boxes))
    return DDHF_ERR_INVALID_ARG;
  if (band_row0[0] != 0 || band_row0[n_bands] != H || comp_off[0] != 0)
    return DDHF_ERR_INVALID_ARG;
  for (int b = 0; b < n_bands; ++b)
    if (band_row0[b + 1] <= band_row0[b] || comp_off[b + 1] < comp_off[b])
      return DDHF_ERR_INVALID_ARG;
  const int64_t nc = comp_off[n_bands];
  if (nc > 0 && !comps) return DDHF_ERR_INVALID_ARG;

  // components by label (labels are sensor linear indices, unique)
  std::vector<int64_t> order((size_t)nc);
  std::iota(order.begin(), order.end(), 0);
  std::sort(order.begin(), order.end(),
            [&](int64_t a, int64_t b) { return comps[a].label < comps[b].label; });
  for (int64_t i = 1; i < nc; ++i)
    if (comps[order[(size_t)i]].label == comps[order[(size_t)i - 1]].label)
      return DDHF_ERR_INVALID_ARG;
  auto index_of = [&](int64_t label) -> int64_t {
    auto it = std::lower_bound(order.begin(), order.end(), label,
                               [&](int64_t i, int64_t l) { return comps[i].label < l; });
    if (it == order.end() || comps[*it].label != label) return -1;
    return *it;
  };

  // join components across every boundary (8-connected neighbours)
  UnionFind uf(nc);
  for (int b = 0; b + 1 < n_bands; ++b) {
    const int32_t *last = edge_labels + (int64_t)b * 2 * W + W;  // band b, last row
    const int32_t *first = edge_labels + (int64_t)(b + 1) * 2 * W;  // band b + 1, first row
    const int64_t off_a = (int64_t)band_row0[b] * W, off_b = (int64_t)band_row0[b + 1] * W;
    for (int x = 0; x < W; ++x) {
      if (last[x] < 0) continue;
      const int64_t ia = index_of(last[x] + off_a);
      if (ia < 0) return DDHF_ERR_INVALID_ARG;
      for (int dx = -1; dx <= 1; ++dx) {
        const int xx = x + dx;
        if (xx < 0 || xx >= W || first[xx] < 0) continue;
        const int64_t ib = index_of(first[xx] + off_b);
        if (ib < 0) return DDHF_ERR_INVALID_ARG;
        uf.unite(ia, ib);
      }
    }
  }
  std::vector<Box5> parts((size_t)nc);
  for (int64_t i = 0; i < nc; ++i)
    parts[(size_t)i] = Box5{comps[i].x0, comps[i].y0, comps[i].x1, comps[i].y1, comps[i].n_px};
  const std::vector<Box5> joined = union_groups(parts, uf);

  // area filter, then Eq. 12 rounds to a fixed point
  std::vector<Box5> cur;
  for (const Box5 &bx : joined)
    if ((int64_t)(bx.x1 - bx.x0 + 1) * (int64_t)(bx.y1 - bx.y0 + 1) >= params->A_min)
      cur.push_back(bx);
  const int64_t B0 = (int64_t)cur.size();
  for (int64_t round = 0; round <= B0 + 1; ++round) {
    UnionFind g((int64_t)cur.size());
    bool any = false;
    for (size_t i = 0; i < cur.size(); ++i)
      for (size_t j = i + 1; j < cur.size(); ++j)
        if (eq12_close(cur[i], cur[j], params->alpha)) {
          any = true;
          g.unite((int64_t)i, (int64_t)j);
        }
    if (!any) break;
    if (round == B0 + 1) return DDHF_ERR_TIMEOUT;  // cannot happen: each round shrinks the list
    cur = union_groups(cur, g);
  }
  std::stable_sort(cur.begin(), cur.end(), [](const Box5 &a, const Box5 &b) {
    if (a.y0 != b.y0) return a.y0 < b.y0;
    if (a.x0 != b.x0) return a.x0 < b.x0;
    if (a.y1 != b.y1) return a.y1 < b.y1;
    if (a.x1 != b.x1) return a.x1 < b.x1;
    return a.n < b.n;
  });
  const int64_t B = (int64_t)cur.size();
  for (int64_t i = 0; i < B && i < cap; ++i)
    boxes[i] = ddhf_box{cur[(size_t)i].x0, cur[(size_t)i].y0, cur[(size_t)i].x1,
                        cur[(size_t)i].y1, cur[(size_t)i].n};
  *n_boxes = (int32_t)B;
  return B > cap ? DDHF_ERR_CAPACITY : DDHF_OK;
}
