// Host-side check of the index arithmetic the sweep kernels use (compiled and
// run by test_geometry_host.py; no GPU needed): for every site of every parity
// and slice, coords_in_slice / cb_index agree, the parity is right, and every
// neighbour index cb_shift(+-mu) is in range and lands on the coordinates
// x +- mu-hat (periodic), and back.  Also the rolling-band order of the
// streaming configuration 12 (stream_band_rank): a permutation of the
// (half-sweep, position) pairs in which every item's three dependencies come
// earlier.
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "lgt_device.cuh"
#include "lgt_internal.h"

using namespace lgt;

static int check(int nt, int n3, int n2, int n1) {
  Geom g;
  g.n1 = n1, g.n2 = n2, g.n3 = n3, g.nt = nt;
  g.half1 = n1 / 2;
  g.vs_half = n1 * n2 * n3 / 2;
  g.vh = g.vs_half * nt;
  const int ext[4] = {nt, n1, n2, n3};  // direction mu = 0: t, 1: x1, 2: x2, 3: x3
  long long checked = 0;
  for (int p = 0; p < 2; p++)
    for (int t = 0; t < nt; t++)
      for (int j = 0; j < g.vs_half; j++) {
        const Coords c = coords_in_slice(g, p, t, j);
        if (c.t != t || c.x1 < 0 || c.x1 >= n1 || c.x2 < 0 || c.x2 >= n2 || c.x3 < 0 || c.x3 >= n3) return 1;
        if (((c.x1 + c.x2 + c.x3 + c.t) & 1) != p) return 2;
        if (cb_index(g, c.x1, c.x2, c.x3, c.t) != t * g.vs_half + j) return 3;
        for (int mu = 0; mu < 4; mu++)
          for (int dir = -1; dir <= 1; dir += 2) {
            const int nb = cb_shift(g, c, mu, dir);
            if (nb < 0 || nb >= g.vh) return 4;
            const int tn = nb / g.vs_half;
            const Coords d = coords_in_slice(g, p ^ 1, tn, nb - tn * g.vs_half);
            int x[4] = {c.t, c.x1, c.x2, c.x3};
            x[mu] = (x[mu] + dir + ext[mu]) % ext[mu];
            if (d.t != x[0] || d.x1 != x[1] || d.x2 != x[2] || d.x3 != x[3]) return 5;
            if (cb_shift(g, d, mu, -dir) != t * g.vs_half + j) return 6;
            checked++;
          }
      }
  printf("dims %d %d %d %d: %lld neighbour relations\n", nt, n3, n2, n1, checked);
  return 0;
}

// every (h, k) ranked once; item (h, slice t) after half-sweep h - 1's items on
// slices t - 1, t, t + 1 (half-sweep h visits slice (h S + k) mod nt at position k)
static int check_band(int nt, int n_half, int D, int S) {
  std::vector<int> seen(nt * n_half, 0);
  std::vector<unsigned> rank_of(nt * n_half);
  for (int h = 0; h < n_half; h++)
    for (int k = 0; k < nt; k++) {
      const unsigned r = stream_band_rank(h, k, nt, n_half, D);
      if (r >= (unsigned)(nt * n_half) || seen[r]++) return 7;
      rank_of[h * nt + k] = r;
    }
  for (int h = 1; h < n_half; h++)
    for (int k = 0; k < nt; k++) {
      const int t = (int)(((long long)h * S + k) % nt);
      for (int d = -1; d <= 1; d++) {
        const int tt = ((t + d) % nt + nt) % nt;
        const int kp = (int)((((long long)tt - (long long)(h - 1) * S) % nt + nt) % nt);  // position of h - 1 on tt
        if (rank_of[(h - 1) * nt + kp] >= rank_of[h * nt + k]) return 8;
      }
    }
  return 0;
}

int main() {
  for (int nt : {2, 4, 6, 12, 32, 96})
    for (int n_half : {1, 2, 5, 20, 64})
      for (int D = 2; D <= nt + 3; D++)
        for (int S = 1; S < D; S++) {
          const int r = check_band(nt, n_half, D, S);
          if (r) {
            printf("FAIL band nt %d n_half %d D %d S %d: check %d\n", nt, n_half, D, S, r);
            return 1;
          }
        }
  const int dims[][4] = {{2, 2, 2, 2}, {4, 6, 10, 14}, {6, 2, 4, 2}, {8, 8, 8, 8}, {2, 4, 2, 6}, {16, 4, 6, 8}, {4, 2, 2, 32}};
  for (const auto &d : dims) {
    const int r = check(d[0], d[1], d[2], d[3]);
    if (r) {
      printf("FAIL dims %d %d %d %d: check %d\n", d[0], d[1], d[2], d[3], r);
      return 1;
    }
  }
  printf("ok\n");
  return 0;
}
