// Runs the oracle's entry points once each on a small state with every shape
// kind, a wall, velocities, both indicators, the box pipeline with the
// contact history, and the gradient, so that a build with AddressSanitizer
// and UndefinedBehaviorSanitizer checks the oracle's memory accesses and
// arithmetic.  Exit status 0 when every call succeeds and every output is
// finite.  Built and run by tests/test_oracle_sanitizers.py (single-threaded,
// without OpenMP).
#include "../oracle/contact_oracle.cpp"

#include <cstdio>

namespace {

bool finite_all(const std::vector<double>& v) {
  for (double x : v)
    if (!std::isfinite(x)) return false;
  return true;
}

int check(const char* what, bool ok) {
  if (!ok) std::fprintf(stderr, "%s failed\n", what);
  return ok ? 0 : 1;
}

}  // namespace

int main() {
  const int n = 4;
  // sphere, cuboid, cube as a 6-plane polytope, a second sphere (on the floor)
  const int32_t type[n] = {0, 1, 2, 0};
  const double param[3 * n] = {6, 0, 0, 4, 3, 5, 0, 0, 0, 5, 0, 0};
  const int32_t foff[n + 1] = {0, 0, 0, 6, 6};
  const double planes[24] = {1, 0, 0, 4, -1, 0, 0, 4, 0, 1, 0, 4, 0, -1, 0, 4, 0, 0, 1, 4, 0, 0, -1, 4};
  const double young[n] = {2, 2, 2, 2}, poisson[n] = {0.3, 0.3, 0.3, 0.3};
  const double pos[3 * n] = {20.3, 20.1, 20.7, 29.0, 21.0, 19.5, 21.0, 29.2, 20.4, 40.2, 40.1, 19.0};
  const double quat[4 * n] = {1, 0, 0, 0, 0.9, 0.1, -0.2, 0.3, 0.8, -0.3, 0.4, 0.1, 1, 0, 0, 0};
  double vel[6 * n];
  for (int k = 0; k < 6 * n; ++k) vel[k] = 0.01 * ((k * 7) % 11 - 5);
  const double walls[4] = {0, 0, -1, -14.5};   // floor: z >= 14.5
  const double wy[1] = {5}, wp[1] = {0.3};
  oracle_config cfg{};
  cfg.n_cells[0] = cfg.n_cells[1] = cfg.n_cells[2] = 64;
  cfg.dx = 1.0;
  cfg.smooth_width = 1.0;
  cfg.damping_c = 0.2;
  cfg.band_eps = 1e-5;
  cfg.n_walls = 1;
  cfg.walls = walls;
  cfg.wall_young = wy;
  cfg.wall_poisson = wp;
  cfg.contact_resolution = 8;
  const int64_t cap = 64;
  std::vector<int32_t> ij(2 * cap), sh(3 * cap), bx(6 * cap), hij(2 * cap);
  std::vector<double> out(11 * cap), aux(11 * cap), f(3 * n), t(3 * n), pc(cap), hc(cap), hb(6 * cap);
  int fails = 0;
  for (int ind = 0; ind < 2; ++ind) {
    cfg.indicator = ind;
    const int64_t P = oracle_contact_step(&cfg, n, type, param, foff, planes, young, poisson, pos, quat, vel, cap,
                                          ij.data(), sh.data(), bx.data(), out.data(), aux.data(), f.data(),
                                          t.data(), 0, nullptr, nullptr, 1);
    fails += check("contact_step", P >= 3 && P <= cap && finite_all(out) && finite_all(f) && finite_all(t));
  }
  std::vector<double> gF(3 * n, 0.5), gT(3 * n, -0.25), gp(3 * n), gq(4 * n);
  fails += check("gradient", oracle_gradient(&cfg, n, type, param, foff, planes, young, poisson, pos, quat, vel,
                                             gF.data(), gT.data(), gp.data(), gq.data(), 1) >= 0 &&
                                 finite_all(gp) && finite_all(gq));
  // the box pipeline with the history over two steps, friction on
  cfg.indicator = 0;
  cfg.box_mode = 1;
  oracle_contact_law law{0.5, 0.5, 0.3, 0.02, 1, 1};
  int64_t nh = 0;
  const int64_t P1 = oracle_contact_step_ext(&cfg, &law, n, type, param, foff, planes, young, poisson, pos, quat,
                                             vel, cap, ij.data(), out.data(), pc.data(), f.data(), t.data(), 0,
                                             nullptr, nullptr, nullptr, cap, hij.data(), hc.data(), hb.data(), &nh,
                                             1);
  fails += check("box step 1", P1 >= 3 && nh >= 1 && finite_all(out));
  std::vector<int32_t> hij2(2 * cap);
  std::vector<double> hc2(cap), hb2(6 * cap);
  int64_t nh2 = 0;
  const int64_t P2 = oracle_contact_step_ext(&cfg, &law, n, type, param, foff, planes, young, poisson, pos, quat,
                                             vel, cap, ij.data(), out.data(), pc.data(), f.data(), t.data(), nh,
                                             hij.data(), hc.data(), hb.data(), cap, hij2.data(), hc2.data(),
                                             hb2.data(), &nh2, 1);
  fails += check("box step 2", P2 == P1 && nh2 >= 1 && finite_all(out) && finite_all(hb2));
  std::vector<int32_t> rough(6 * cap);
  std::vector<double> boxes(6 * cap), flags(2 * cap);
  fails += check("box_pipeline", oracle_box_pipeline(&cfg, n, type, param, foff, planes, young, poisson, pos, quat,
                                                     nh, hij.data(), hb.data(), cap, rough.data(), boxes.data(),
                                                     flags.data()) == P1);
  double c[3];
  fails += check("centroid", oracle_polytope_centroid(planes, 6, c) == 0 && std::fabs(c[0]) < 1e-12);
  std::vector<double> shift(3 * n);
  fails += check("shift", oracle_polytope_shift(&cfg, n, type, param, foff, planes, young, poisson, pos, quat,
                                                shift.data()) == 0);
  std::printf("oracle sanitizer run: %d failures\n", fails);
  return fails == 0 ? 0 : 1;
}
