// Droplet statistics of a density field (host code): condensate on the walls of the
// channel of Section 3.3, measured as in the reading of the droplet measure (liquid
// nodes above a density threshold, droplets as 8-connected liquid components that
// touch a wall, spacing of their centroids along each wall, condensed mass).
#include <algorithm>
#include <cmath>
#include <cstddef>
#include <vector>

#include "../../include/lbm.h"

namespace {

// union-find over node indices with path halving
struct Components {
  std::vector<int> parent;
  explicit Components(size_t n) : parent(n) {
    for (size_t i = 0; i < n; i++) parent[i] = (int)i;
  }
  int find(int a) {
    while (parent[a] != a) {
      parent[a] = parent[parent[a]];
      a = parent[a];
    }
    return a;
  }
  void unite(int a, int b) {
    a = find(a);
    b = find(b);
    if (a != b) parent[std::max(a, b)] = std::min(a, b);
  }
};

struct Blob {
  double sx = 0.0, sc = 0.0, ss = 0.0;  // sum of x, of cos and sin of the x phase
  long n = 0;
  bool bottom = false, top = false;
};

}  // namespace

extern "C" int lbm_droplet_stats(const double *rho, int nx, int ny, double threshold,
                                 double rho_v, int periodic_x, lbm_droplet_stats_t *out) {
  if (!rho || !out || nx < 1 || ny < 1 || nx > (1 << 20) || ny > (1 << 20)) return LBM_ERR_ARG;
  if ((long long)nx * ny > (1LL << 31) - 1 || !(threshold == threshold)) return LBM_ERR_ARG;
  const size_t n = (size_t)nx * ny;
  std::vector<unsigned char> liq(n);
  double mass = 0.0;
  long nliq = 0;
  for (size_t k = 0; k < n; k++) {
    liq[k] = rho[k] > threshold;
    if (liq[k]) {
      mass += rho[k] - rho_v;
      nliq++;
    }
  }
  // 8-connected components: join each liquid node with its liquid neighbours to the
  // right and in the row above (left, above-left and above-right), x wrapping when periodic
  Components cc(n);
  for (int y = 0; y < ny; y++)
    for (int x = 0; x < nx; x++) {
      const int id = y * nx + x;
      if (!liq[id]) continue;
      const int dxs[4] = {1, -1, 0, 1}, dys[4] = {0, 1, 1, 1};
      for (int d = 0; d < 4; d++) {
        int xs = x + dxs[d];
        const int ys = y + dys[d];
        if (ys >= ny) continue;
        if (xs < 0 || xs >= nx) {
          if (!periodic_x || nx < 2) continue;
          xs = (xs + nx) % nx;
        }
        const int nb = ys * nx + xs;
        if (liq[nb]) cc.unite(id, nb);
      }
    }
  std::vector<int> slot(n, -1);
  std::vector<Blob> blobs;
  const double kTwoPi = 6.283185307179586476925286766559;
  for (int y = 0; y < ny; y++)
    for (int x = 0; x < nx; x++) {
      const int id = y * nx + x;
      if (!liq[id]) continue;
      const int r = cc.find(id);
      if (slot[r] < 0) {
        slot[r] = (int)blobs.size();
        blobs.emplace_back();
      }
      Blob &b = blobs[slot[r]];
      b.n++;
      b.sx += x;
      b.sc += std::cos(kTwoPi * x / nx);
      b.ss += std::sin(kTwoPi * x / nx);
      if (y == 0) b.bottom = true;
      if (y == ny - 1) b.top = true;
    }
  lbm_droplet_stats_t s{};
  std::vector<double> cx[2];
  for (const Blob &b : blobs) {
    double c = b.sx / (double)b.n;
    if (periodic_x) {  // circular mean of the x positions
      double a = std::atan2(b.ss, b.sc);
      if (a < 0.0) a += kTwoPi;
      c = a * nx / kTwoPi;
    }
    if (b.bottom) cx[0].push_back(c);
    if (b.top) cx[1].push_back(c);
    if (!b.bottom && !b.top) s.detached++;
  }
  for (int w = 0; w < 2; w++) {
    s.count[w] = (int)cx[w].size();
    if (cx[w].size() >= 2) {
      std::sort(cx[w].begin(), cx[w].end());
      s.spacing[w] = periodic_x ? (double)nx / (double)cx[w].size()
                                : (cx[w].back() - cx[w].front()) / (double)(cx[w].size() - 1);
    }
  }
  s.condensed_mass = mass;
  s.liquid_nodes = (long long)nliq;
  *out = s;
  return LBM_OK;
}
