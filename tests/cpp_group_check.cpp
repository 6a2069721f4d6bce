// Host checks of the momentum-sector group construction (csrc/hub_group.h), no GPU:
// closure and refusals, the action on spin strings as a representation with fermion signs
// (against a swap count), orbits and stabilisers, and every move-table entry against the action.
// Exit status = number of failed checks.
#include <cstdio>
#include <numeric>
#include <random>
#include <string>
#include <vector>

#include "hub_group.h"

using namespace hub;

static int failures = 0;
#define CHECK(c)                                                         \
  do {                                                                   \
    if (!(c)) {                                                          \
      ++failures;                                                        \
      std::printf("FAIL line %d: %s\n", __LINE__, #c);                   \
    }                                                                    \
  } while (0)

// sign of reordering the images of the occupied sites, by counting the swaps of a bubble sort
static int swap_sign(const std::vector<int> &perm, uint32_t x) {
  std::vector<int> img;
  for (int i = 0; i < (int)perm.size(); ++i)
    if ((x >> i) & 1u) img.push_back(perm[i]);
  int swaps = 0;
  for (size_t a = 0; a < img.size(); ++a)
    for (size_t b = 0; b + 1 < img.size() - a; ++b)
      if (img[b] > img[b + 1]) {
        std::swap(img[b], img[b + 1]);
        ++swaps;
      }
  return (swaps & 1) ? -1 : 1;
}

static std::vector<int32_t> chain(int M) {
  std::vector<int32_t> p(M);
  for (int i = 0; i < M; ++i) p[i] = (i + M - 1) % M;
  return p;
}

static std::vector<int32_t> torus(int Lx, int Ly) {
  std::vector<int32_t> p(2 * Lx * Ly);
  for (int y = 0; y < Ly; ++y)
    for (int x = 0; x < Lx; ++x) {
      p[x + Lx * y] = (x + Lx - 1) % Lx + Lx * y;
      p[Lx * Ly + x + Lx * y] = x + Lx * ((y + Ly - 1) % Ly);
    }
  return p;
}

static void check_group(const Group &G, int N) {
  const int g = G.g, M = G.M;
  std::mt19937 rng(7);
  const std::vector<uint32_t> S = strings_of(M, N);
  for (int trial = 0; trial < 200 && !S.empty(); ++trial) {
    const uint32_t x = S[rng() % S.size()];
    for (int a = 0; a < g; ++a) {
      int sa;
      const uint32_t ya = group_act(G, a, x, &sa);
      CHECK(sa == swap_sign(G.perm[a], x));
      CHECK(__builtin_popcount(ya) == N);
      for (int b = 0; b < g; b += 3) {
        int sb, sab;
        const uint32_t yb = group_act(G, b, ya, &sb);
        const uint32_t yab = group_act(G, G.mul[(size_t)a * g + b], x, &sab);
        CHECK(yb == yab && sa * sb == sab);   // a representation, signs included
      }
    }
  }
  // orbits: |orbit| |stabiliser| = |G|, the stabiliser closed under products
  for (uint32_t x : S) {
    const OrbitOf o = orbit_of(G, x);
    std::vector<uint32_t> images;
    for (int e = 0; e < g; ++e) {
      int s;
      images.push_back(group_act(G, e, x, &s));
    }
    std::sort(images.begin(), images.end());
    const size_t orbit = (size_t)(std::unique(images.begin(), images.end()) - images.begin());
    CHECK(orbit * o.stab.size() == (size_t)g);
    CHECK(o.least == images[0]);
    for (const auto &h1 : o.stab)
      for (const auto &h2 : o.stab) {
        const int p = G.mul[(size_t)h1.first * g + h2.first];
        bool in = false;
        for (const auto &h : o.stab) in = in || (h.first == p && h.second == h1.second * h2.second);
        CHECK(in);
      }
  }
  // columns: every string once; each table entry agrees with the action
  Columns C;
  std::string err;
  CHECK(build_columns(G, S, &C, &err) == 0);
  CHECK(C.cbits.size() == S.size());
  for (size_t c = 0; c < C.cbits.size(); ++c) {
    const int k = (int)(C.cinfo[c] & 0xff), type = (int)((C.cinfo[c] >> 8) & 0xff);
    const int off = C.tab_off[2 * type], bs = C.tab_off[2 * type + 1];
    for (int e = 0; e < g; ++e) {
      const uint16_t w = C.tab[off + e * bs + k];
      const size_t c2 = c - k + (w & 0xff);
      const int sig = (w & 0x8000) ? -1 : 1;
      int s;
      const uint32_t d = group_act(G, e, C.cbits[c], &s);   // e c_k |R> = csign[c] s |d>
      CHECK(c2 < C.cbits.size() && d == C.cbits[c2]);
      CHECK(C.csign[c] * s == sig * C.csign[c2]);
    }
  }
}

int main() {
  std::string err;
  Group G;
  // chain: k = 0 and k = pi, -1 refused at odd M
  for (int M : {1, 2, 5, 6, 8}) {
    const std::vector<int32_t> p = chain(M);
    const int32_t plus = 1, minus = -1;
    CHECK(make_group(M, 1, p.data(), &plus, &G, &err) == 0 && G.g == M);
    for (int N = 0; N <= M; ++N) check_group(G, N);
    CHECK((make_group(M, 1, p.data(), &minus, &G, &err) == 0) == (M % 2 == 0));
  }
  // tori
  {
    const std::vector<int32_t> p = torus(4, 4);
    const int32_t ch[2] = {-1, 1};
    CHECK(make_group(16, 2, p.data(), ch, &G, &err) == 0 && G.g == 16);
    for (int N : {0, 3, 8}) check_group(G, N);
    const std::vector<int32_t> q = torus(3, 2);
    const int32_t bad[2] = {-1, 1}, good[2] = {1, -1};
    CHECK(make_group(6, 2, q.data(), bad, &G, &err) == 3);
    CHECK(make_group(6, 2, q.data(), good, &G, &err) == 0 && G.g == 6);
    for (int N : {2, 3}) check_group(G, N);
  }
  // a translation with a reflection: not abelian
  {
    std::vector<int32_t> p = torus(3, 3);
    for (int y = 0; y < 3; ++y) {
      p[9 + 0 + 3 * y] = 1 + 3 * y;
      p[9 + 1 + 3 * y] = 0 + 3 * y;
      p[9 + 2 + 3 * y] = 2 + 3 * y;
    }
    const int32_t ch[2] = {1, 1};
    CHECK(make_group(9, 2, p.data(), ch, &G, &err) == 2);
  }
  // more than 64 elements: two independent cycles of lengths 7 and 11 on 18 sites
  {
    std::vector<int32_t> p(2 * 18);
    for (int i = 0; i < 18; ++i) {
      p[i] = i < 7 ? (i + 1) % 7 : i;
      p[18 + i] = i >= 7 ? 7 + (i - 7 + 1) % 11 : i;
    }
    const int32_t ch[2] = {1, 1};
    CHECK(make_group(18, 2, p.data(), ch, &G, &err) == 1);
  }
  std::printf("%s: %d failure(s)\n", failures ? "FAIL" : "ok", failures);
  return failures;
}
