// Seeded synthetic networks inside the library (sm_synth_network,
// sm_net_build_synthetic).
//
// The paper's network (UMIST rate12, 468 species x 6175 reactions, Section 3)
// is not distributed with the library, so networks of its shape are drawn
// from H, C, O and e-: species are neutral, cationic and small anionic
// C_c H_h O_o compositions (small ones first) named by formula and stored in
// alphabetical order; reactions come grouped by class, 60 % two-body, 20 %
// cosmic-ray, 15 % photo and 5 % dissociative recombination, with 1-2
// reactants and 1-4 products that conserve every element and the charge; the
// rate parameters are drawn per class.  Every decision is integer arithmetic on
// counter-based SplitMix64 words (Steele, Lea & Flood 2014), so the arrays are
// the same on every platform and equal, element for element, to those of the
// package's Python input generator (synth/network.py) for the same seed, which
// the tests check.  Only inputs are produced here: S, the formats and the rest
// of the method are built from these arrays by sm_net_build.
#include <algorithm>
#include <array>
#include <cmath>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "internal.h"

namespace {

constexpr uint64_t kGolden = 0x9E3779B97F4A7C15ull;

uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

uint64_t stream_key(uint64_t seed, uint64_t stream) { return mix64(seed ^ mix64(stream * 0xD1B54A32D192ED03ull)); }

struct Stream {
  uint64_t key, i = 0;
  explicit Stream(uint64_t k) : key(k) {}
  uint64_t next() { return mix64(key + (++i) * kGolden); }
  double uniform() { return (double)(next() >> 11) * (1.0 / 9007199254740992.0); }
  // integer in [0, n) by 32 x 32 multiply-shift (n < 2^32)
  uint64_t below(uint64_t n) { return ((next() >> 32) * n) >> 32; }
  int weighted(const std::vector<int64_t>& w) {
    int64_t total = 0;
    for (int64_t v : w) total += v;
    const int64_t r = (int64_t)below((uint64_t)total);
    int64_t acc = 0;
    for (size_t k = 0; k < w.size(); ++k) {
      acc += w[k];
      if (r < acc) return (int)k;
    }
    return (int)w.size() - 1;
  }
};

using Comp = std::array<int32_t, 4>;   // (H, C, O, charge)

std::string formula(const Comp& s) {
  const int h = s[0], c = s[1], o = s[2], q = s[3];
  if (h == 0 && c == 0 && o == 0) return "E-";
  std::string out;
  const std::pair<const char*, int> parts[3] = {{"C", c}, {"H", h}, {"O", o}};
  for (const auto& pr : parts) {
    if (pr.second == 1) out += pr.first;
    else if (pr.second > 1) out += std::string(pr.first) + std::to_string(pr.second);
  }
  return out + (q > 0 ? "+" : q < 0 ? "-" : "");
}

int hub_weight(const std::string& name) {
  static const std::map<std::string, int> w = {{"H", 62}, {"H2", 28}, {"H+", 8}, {"H3+", 8}, {"C+", 6},
                                               {"O", 6},  {"C", 5},   {"O+", 3}, {"CO", 4},  {"OH", 4},
                                               {"H2O", 3}, {"CH", 3},  {"H2+", 3}};
  auto it = w.find(name);
  return it == w.end() ? 1 : it->second;
}

struct Generator {
  int32_t n_s, n_r;
  std::vector<Comp> comp;
  std::vector<std::string> names;
  std::map<Comp, int> by_comp;
  std::vector<int64_t> n_atoms, w_hub, ones;
  std::vector<char> heavy, small, cation;
  int e_idx = -1;
  Stream rr{0};
  std::vector<std::vector<int>> reac_l, prod_l;
  std::vector<int8_t> cls_l;
  std::map<std::pair<std::vector<int>, std::vector<int>>, char> seen;

  // First index whose running sum of the masked weights exceeds a draw below
  // their total; -1 when nothing is eligible.
  int pick(const std::vector<char>& mask, const std::vector<int64_t>& w) {
    std::vector<int64_t> cum(n_s);
    int64_t acc = 0;
    for (int i = 0; i < n_s; ++i) {
      acc += mask[i] ? w[i] : 0;
      cum[i] = acc;
    }
    if (acc == 0) return -1;
    const int64_t r = (int64_t)rr.below((uint64_t)acc);
    return (int)(std::upper_bound(cum.begin(), cum.end(), r) - cum.begin());
  }

  // Split `total` into m existing species; the last one found by lookup.
  bool decompose(Comp rem, int m, std::vector<int>& out) {
    out.clear();
    for (int i = 0; i < m - 1; ++i) {
      const int left = m - 1 - i;
      const int64_t rem_atoms = (int64_t)rem[0] + rem[1] + rem[2];
      std::vector<char> fits(n_s);
      for (int p = 0; p < n_s; ++p)
        fits[p] = comp[p][0] <= rem[0] && comp[p][1] <= rem[1] && comp[p][2] <= rem[2] && small[p] &&
                  rem_atoms - n_atoms[p] >= left - 1;
      const int p = pick(fits, w_hub);
      if (p < 0) return false;
      out.push_back(p);
      for (int e = 0; e < 4; ++e) rem[e] -= comp[p][e];
    }
    auto it = by_comp.find(rem);
    if (it == by_comp.end()) return false;
    out.push_back(it->second);
    return true;
  }

  bool accept(std::vector<int> reac, std::vector<int> prods, int8_t cls) {
    std::sort(reac.begin(), reac.end());
    std::sort(prods.begin(), prods.end());
    if (reac == prods) return false;
    auto key = std::make_pair(reac, prods);
    if (seen.count(key)) return false;
    seen[key] = 1;
    reac_l.push_back(reac);
    prod_l.push_back(prods);
    cls_l.push_back(cls);
    return true;
  }

  bool draw(int8_t cls) {
    const std::vector<int64_t> m_two = {5, 65, 22, 8}, m_diss = {70, 25, 5}, m_dr = {70, 30};
    std::vector<int> prods;
    for (int attempt = 0; attempt < 500; ++attempt) {
      if (cls == SM_TWO_BODY) {
        const int a = pick(heavy, ones), b = pick(heavy, w_hub);
        Comp tot;
        for (int e = 0; e < 4; ++e) tot[e] = comp[a][e] + comp[b][e];
        const int m = 1 + rr.weighted(m_two);
        if (decompose(tot, m, prods) && accept({a, b}, prods, cls)) return true;
      } else if (cls == SM_COSMIC_RAY || cls == SM_PHOTO) {
        const int a = pick(heavy, ones);
        Comp ion = comp[a];
        ion[3] += 1;
        bool ok;
        if (rr.below(100) < 45 && by_comp.count(ion)) {
          prods = {by_comp[ion], e_idx};
          ok = true;
        } else {
          const int m = 2 + rr.weighted(m_diss);
          ok = decompose(comp[a], m, prods);
        }
        if (ok && accept({a}, prods, cls)) return true;
      } else {
        const int a = pick(cation, ones);
        Comp tot;
        for (int e = 0; e < 4; ++e) tot[e] = comp[a][e] + comp[e_idx][e];
        const int m = n_atoms[a] == 1 ? 1 : 2 + rr.weighted(m_dr);
        if (decompose(tot, m, prods) && accept({a, e_idx}, prods, cls)) return true;
      }
    }
    return false;
  }
};

}  // namespace

extern "C" sm_status sm_synth_network(uint64_t seed, int32_t n_s, int32_t n_r, int32_t* comp_out,
                                      int32_t* reactants, int32_t* products, int8_t* rclass, double* alpha,
                                      double* beta, double* gamma) {
  if (n_s < 12 || n_r < 1 || !comp_out || !reactants || !products || !rclass || !alpha || !beta || !gamma)
    return SM_EINVAL;
  // species pool in a fixed order, each with one jitter draw
  std::vector<Comp> pool;
  for (int c = 0; c <= 8; ++c)
    for (int o = 0; o <= 4; ++o)
      for (int h = 0; h <= 10; ++h) {
        const int n_at = h + c + o;
        if (n_at == 0 || n_at > 14) continue;
        for (int q : {0, 1, -1}) {
          if (q == -1 && n_at > 3) continue;
          pool.push_back({h, c, o, q});
        }
      }
  if ((int64_t)pool.size() < (int64_t)n_s - 1) return SM_EINVAL;
  const std::vector<Comp> mandatory = {{1, 0, 0, 0}, {1, 0, 0, 1}, {2, 0, 0, 0}, {0, 1, 0, 0}, {0, 1, 0, 1},
                                       {0, 0, 1, 0}, {0, 0, 1, 1}, {2, 0, 0, 1}, {3, 0, 0, 1}, {1, 0, 0, -1}};
  Stream rs(stream_key(seed, 1));
  std::vector<std::pair<int64_t, Comp>> keyed;
  for (const Comp& sp : pool) {
    const int h = sp[0], c = sp[1], o = sp[2], q = sp[3];
    const int64_t size = h + 2 * (c + o) + (q != 0 ? 1 : 0) + (q < 0 ? 2 : 0);
    const int64_t jitter = (int64_t)rs.below(1u << 20);
    const bool mand = std::find(mandatory.begin(), mandatory.end(), sp) != mandatory.end();
    keyed.push_back({mand ? -(int64_t(1) << 40) : (size << 22) + jitter, sp});
  }
  std::sort(keyed.begin(), keyed.end());
  std::vector<Comp> chosen;
  for (int i = 0; i < n_s - 1; ++i) chosen.push_back(keyed[i].second);
  chosen.push_back({0, 0, 0, -1});
  std::vector<int> order(n_s);
  for (int i = 0; i < n_s; ++i) order[i] = i;
  std::vector<std::string> nm(n_s);
  for (int i = 0; i < n_s; ++i) nm[i] = formula(chosen[i]);
  std::sort(order.begin(), order.end(), [&](int a, int b) { return nm[a] < nm[b]; });

  Generator g;
  g.n_s = n_s;
  g.n_r = n_r;
  for (int i = 0; i < n_s; ++i) {
    g.comp.push_back(chosen[order[i]]);
    g.names.push_back(nm[order[i]]);
  }
  for (int i = 0; i < n_s; ++i) g.by_comp[g.comp[i]] = i;
  g.n_atoms.resize(n_s);
  g.w_hub.resize(n_s);
  g.ones.assign(n_s, 1);
  g.heavy.resize(n_s);
  g.small.resize(n_s);
  g.cation.resize(n_s);
  for (int i = 0; i < n_s; ++i) {
    g.n_atoms[i] = (int64_t)g.comp[i][0] + g.comp[i][1] + g.comp[i][2];
    g.w_hub[i] = hub_weight(g.names[i]);
    g.heavy[i] = g.n_atoms[i] >= 1;
    g.small[i] = g.n_atoms[i] >= 1 && g.n_atoms[i] <= 3;
    g.cation[i] = g.comp[i][3] == 1 && g.heavy[i];
    if (g.names[i] == "E-") g.e_idx = i;
  }
  g.w_hub[g.e_idx] = 0;
  g.rr = Stream(stream_key(seed, 2));
  const int32_t n2 = n_r * 60 / 100, ncr = n_r * 20 / 100, nph = n_r * 15 / 100, ndr = n_r - n2 - ncr - nph;
  const std::pair<int8_t, int32_t> plan[4] = {
      {SM_TWO_BODY, n2}, {SM_COSMIC_RAY, ncr}, {SM_PHOTO, nph}, {SM_DISS_RECOMB, ndr}};
  for (const auto& pc : plan)
    for (int32_t t = 0; t < pc.second; ++t)
      if (!g.draw(pc.first)) return SM_EINVAL;   // network too small for its reaction count

  for (int i = 0; i < n_s; ++i)
    for (int e = 0; e < 4; ++e) comp_out[4 * i + e] = g.comp[i][e];
  for (int32_t j = 0; j < n_r; ++j) {
    for (int e = 0; e < 2; ++e) reactants[2 * j + e] = e < (int)g.reac_l[j].size() ? g.reac_l[j][e] : -1;
    for (int e = 0; e < 4; ++e) products[4 * j + e] = e < (int)g.prod_l[j].size() ? g.prod_l[j][e] : -1;
    rclass[j] = g.cls_l[j];
  }
  Stream rp(stream_key(seed, 3));
  for (int32_t j = 0; j < n_r; ++j) {
    const double u1 = rp.uniform(), u2 = rp.uniform(), u3 = rp.uniform();
    const int c = rclass[j];
    beta[j] = 0.0;
    gamma[j] = 0.0;
    if (c == SM_TWO_BODY || c == SM_DISS_RECOMB) {
      alpha[j] = std::pow(10.0, -12.0 + 3.0 * u1);
      beta[j] = -1.0 + 2.0 * u2;
      gamma[j] = 500.0 * u3;
    } else if (c == SM_COSMIC_RAY) {
      alpha[j] = std::pow(10.0, 3.0 * u1);
    } else {
      alpha[j] = std::pow(10.0, -11.0 + 2.0 * u1);
      gamma[j] = 1.0 + 2.0 * u3;
    }
  }
  return SM_OK;
}

extern "C" sm_status sm_net_build_synthetic(uint64_t seed, int32_t n_s, int32_t n_r, int32_t device,
                                            sm_net** out) {
  if (!out || n_s < 12 || n_r < 1) return SM_EINVAL;
  std::vector<int32_t> comp(4 * (size_t)n_s), reac(2 * (size_t)n_r), prod(4 * (size_t)n_r);
  std::vector<int8_t> cls(n_r);
  std::vector<double> alpha(n_r), beta(n_r), gamma(n_r);
  sm_status st = sm_synth_network(seed, n_s, n_r, comp.data(), reac.data(), prod.data(), cls.data(),
                                  alpha.data(), beta.data(), gamma.data());
  if (st != SM_OK) return st;
  sm_net_desc d{n_s, n_r, 3, comp.data(), reac.data(), prod.data(), cls.data(), alpha.data(), beta.data(),
                gamma.data()};
  return sm_net_build(&d, device, out);
}
