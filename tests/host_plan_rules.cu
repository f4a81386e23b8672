// Host-only checks of the launch planning in qap_host.cuh (no GPU, no CUDA
// calls): every plan the rules choose holds n, fits the shared memory it is
// given, is one the library compiles, and follows the preferences the rules
// state.  Built and run by tests/test_host_plans.py; prints "ok" and exits 0,
// or prints the first violations and exits 1.
#include <cstdio>
#include <random>
#include <vector>

#include "../paper_2307_11248_gb300/csrc/qap_host.cuh"

using qaph::Plan;

namespace {

int fails = 0;

void fail(const char* what, int n, int threads, int many, const Plan& p) {
  if (fails++ < 10)
    std::printf("FAIL %s: n=%d threads=%d many=%d -> (%d, %d, %d)\n", what, n, threads, many,
                p.nt, p.maxpt, p.store);
}

bool compiled_register_plan(const Plan& p) {
  for (const Plan& q : qaph::kPlans)
    if (q.nt == p.nt && q.maxpt == p.maxpt && q.store == 0) return true;
  return false;
}

bool fits(int n, const Plan& p) { return qapk::row_segments(n, p.maxpt) <= p.nt; }

// The rules of choose_plan on their own.
void check_choose_plan() {
  for (int n = 2; n <= 181; ++n)
    for (int threads : {0, 128, 256, 512, 1024})
      for (int many = 0; many < 2; ++many) {
        Plan p{};
        const bool ok = qaph::choose_plan(n, threads, many != 0, &p);
        if (threads == 0 && !ok) fail("no automatic plan", n, threads, many, p);
        if (!ok) {
          // a fixed thread count may be too small for n, never too large
          for (const Plan& q : qaph::kPlans)
            if (q.nt == threads && fits(n, q)) fail("fixed count refused", n, threads, many, q);
          continue;
        }
        if (!compiled_register_plan(p)) fail("not a compiled plan", n, threads, many, p);
        if (!fits(n, p)) fail("plan does not hold n", n, threads, many, p);
        // the fewest slots that fit for its thread count
        for (const Plan& q : qaph::kPlans)
          if (q.nt == p.nt && q.maxpt < p.maxpt && fits(n, q))
            fail("not the fewest slots", n, threads, many, p);
        if (threads != 0) {
          if (p.nt != threads) fail("fixed count not kept", n, threads, many, p);
          continue;
        }
        // automatic: 256 threads with more than 8 slots only with many walks
        if (!many && p.nt == 256 && p.maxpt > 8) fail("256 wide without walks", n, 0, many, p);
        // a preferred plan with fewer threads is never passed over
        for (int nt : {128, 256, 512, 1024}) {
          if (nt >= p.nt) break;
          Plan q{};
          if (qaph::plan_for(n, nt, &q) &&
              (q.maxpt <= 8 || nt == 512 || (many && nt == 256)))
            fail("a preferred plan with fewer threads fits", n, 0, many, p);
        }
        // with many walks a 256-thread plan is taken wherever one fits and
        // 128 threads with at most 8 slots do not
        Plan q128{}, q256{};
        const bool f128 = qaph::plan_for(n, 128, &q128) && q128.maxpt <= 8;
        if (many && !f128 && qaph::plan_for(n, 256, &q256) && p.nt != 256)
          fail("256 threads passed over with many walks", n, 0, many, p);
      }
}

// wide_flows: flows up to 3000 (int16 elements); big_dist: distances up to
// 30000 (beyond int8: the int64 element path)
qaph::DevInstance make_instance(int n, bool symmetric, bool wide_flows, bool big_dist,
                                unsigned seed, int* fbytes, int dbytes) {
  std::mt19937 rng(seed);
  std::vector<int64_t> F((size_t)n * n, 0), D((size_t)n * n, 0);
  const int fmax = wide_flows ? 3000 : 99;
  const int dmax = big_dist ? 30000 : 99;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      if (i == j || (symmetric && j < i)) continue;
      F[(size_t)i * n + j] = rng() % (fmax + 1);
      D[(size_t)i * n + j] = rng() % (dmax + 1);
      if (symmetric) {
        F[(size_t)j * n + i] = F[(size_t)i * n + j];
        D[(size_t)j * n + i] = D[(size_t)i * n + j];
      }
    }
  qaph::DevInstance di;
  if (qaph::inspect_instance(F.data(), D.data(), n, &di) != QAP_OK) std::printf("inspect failed\n");
  if (di.wide != (big_dist ? 1 : 0)) std::printf("FAIL element path of n=%d\n", n), ++fails;
  *fbytes = qaph::flow_bytes(di, dbytes);
  di.ldF = qaph::pad_ldF(n, *fbytes);
  di.ldP = qaph::pad_ldP(n, qaph::pbytes_of(*fbytes));
  return di;
}

// choose_plan_fit on instances of every kind, with the shared memory of a
// GB300 (227 KB per CTA) and the batch kernel's reserve.
void check_choose_plan_fit() {
  const int optin = 232448;
  for (int n = 2; n <= 256; n += (n < 40 ? 1 : 3))
    for (int kind = 0; kind < 8; ++kind) {
      const bool sym = kind & 1, wide = (kind >> 1) == 1, i64 = (kind >> 1) >= 2;
      const bool big = (kind >> 1) == 3;
      const int dbytes = i64 ? 8 : 4;
      int fbytes = 0;
      const qaph::DevInstance di = make_instance(n, sym, wide, big, 1000u + n * 7 + kind,
                                                 &fbytes, dbytes);
      for (int reserve : {0, 16})
        for (int form : {QAP_PHASE_X_AUTO, QAP_PHASE_X_DOTS})
        for (int many = 0; many < 2; ++many) {
          Plan p{};
          if (!qaph::choose_plan_fit(n, 0, many != 0, &di, 1, fbytes, dbytes, optin, reserve,
                                     form, &p)) {
            fail("no plan fits", n, 0, many, p);
            continue;
          }
          const int smem = qaph::plan_smem(p, &di, 1, fbytes, dbytes);
          if (smem + reserve > optin) fail("shared memory exceeded", n, 0, many, p);
          if (fbytes == 8) {
            // int64 elements: F always global, P global only where it does
            // not fit, no products form; the workspace plan only beyond the
            // register plans
            if (!(p.store & qapk::kGlobalFlow)) fail("int64 flows not global", n, 0, many, p);
            if (p.store & qapk::kProductM) fail("products form on int64", n, 0, many, p);
            if (p.store & qapk::kGlobalP) {
              Plan q = p;
              q.store &= ~qapk::kGlobalP;
              if (qaph::plan_smem(q, &di, 1, fbytes, dbytes) + reserve <= optin)
                fail("P global where it fits", n, 0, many, p);
            }
            if (!fits(n, p)) fail("plan does not hold n", n, 0, many, p);
            if (p.store & qapk::kGlobalDelta) {
              if (p.nt != qaph::kLargePlan.nt || p.maxpt != qaph::kLargePlan.maxpt)
                fail("not the large plan", n, 0, many, p);
              if (n <= 181) fail("int64 workspace plan within the register plans", n, 0, many, p);
            } else {
              if (n > 181) fail("register plan beyond 181", n, 0, many, p);
              if (!compiled_register_plan(Plan{p.nt, p.maxpt, 0}))
                fail("not a compiled plan", n, 0, many, p);
            }
            continue;
          }
          if (p.store & qapk::kGlobalP) fail("P global on a narrow path", n, 0, many, p);
          const int base = p.store & ~(qapk::kProductM | qapk::kNoTransposed);
          if (base != 0) {
            // the workspace plan: beyond the register plans' n, or where the
            // register plan the rules pick without the two-walks preference
            // (its fallback) does not fit shared memory
            if (!(p.store & qapk::kGlobalDelta))
              fail("flows global without workspace", n, 0, many, p);
            if (p.nt != qaph::kLargePlan.nt || p.maxpt != qaph::kLargePlan.maxpt)
              fail("not the large plan", n, 0, many, p);
            if (!fits(n, p)) fail("large plan does not hold n", n, 0, many, p);
            Plan r{};
            if (n <= 181 && qaph::choose_plan(n, 0, false, &r) &&
                qaph::plan_smem(r, &di, 1, fbytes, dbytes) + reserve <= optin)
              fail("workspace plan where a register plan fits", n, 0, many, p);
            if ((p.store & qapk::kGlobalFlow) &&
                qaph::plan_smem(qaph::kLargePlan, &di, 1, fbytes, dbytes) + reserve <= optin)
              fail("flows in global memory where they fit", n, 0, many, p);
            continue;
          }
          if (n > 181) fail("register plan beyond 181", n, 0, many, p);
          const Plan reg{p.nt, p.maxpt, 0};
          if (!compiled_register_plan(reg)) fail("not a compiled plan", n, 0, many, p);
          if (!fits(n, p)) fail("plan does not hold n", n, 0, many, p);
          // the products form with the transposed copies where it fits, else
          // without them where compiled and fitting, else the dot products
          const bool two = many && p.nt == 256 && p.maxpt > 8;
          auto fits_as = [&](int store) {
            Plan m = reg;
            m.store = store;
            const int ms = qaph::plan_smem(m, &di, 1, fbytes, dbytes);
            return ms + reserve <= optin && (!two || 2 * (ms + reserve + 1024) <= optin + 1024);
          };
          const int pm = qapk::kProductM, pn = qapk::kProductM | qapk::kNoTransposed;
          if (p.store & qapk::kProductM) {
            if (fbytes == 8 || form == QAP_PHASE_X_DOTS)
              fail("products form where it does not apply", n, 0, many, p);
            if (!qaph::has_product_form(reg, fbytes)) fail("products form not compiled", n, 0, many, p);
            if (p.store & qapk::kNoTransposed) {
              if (!qaph::has_notrans_form(reg, fbytes)) fail("no-transposes form not compiled", n, 0, many, p);
              if (fits_as(pm)) fail("transposes left out where they fit", n, 0, many, p);
            }
          } else if (p.store & qapk::kNoTransposed) {
            fail("no-transposes bit without products", n, 0, many, p);
          } else if (form == QAP_PHASE_X_AUTO && fbytes != 8 && qaph::has_product_form(reg, fbytes)) {
            if (fits_as(pm) || (qaph::has_notrans_form(reg, fbytes) && fits_as(pn)))
              fail("products form left out where it fits", n, 0, many, p);
          }
          if (p.nt == 256 && p.maxpt > 8) {
            if (!many) fail("256 wide without walks", n, 0, many, p);
            if (2 * (smem + reserve + 1024) > optin + 1024)
              fail("two CTAs per SM do not fit", n, 0, many, p);
          }
        }
    }
}

}  // namespace

// The admission of an instance to an element path (no GPU): the narrow
// path holds every dot-product sum of 2n element products below 2^31, so
// the int16-flow extremes F = -32768, D = -128 are narrow up to n = 255 and
// wide at n = 256; the int64 path stops where the bound B reaches 2^62.
void check_admission() {
  auto admit = [](int n, int64_t f, int64_t d, qaph::DevInstance* di) {
    std::vector<int64_t> F((size_t)n * n, f), D((size_t)n * n, d);
    return qaph::inspect_instance(F.data(), D.data(), n, di);
  };
  qaph::DevInstance di;
  if (admit(255, -32768, -128, &di) != QAP_OK || di.wide) fail("n=255 extremes", 255, 0, 0, {});
  if (admit(256, -32768, -128, &di) != QAP_OK || !di.wide) fail("n=256 extremes", 256, 0, 0, {});
  if (admit(20, 32767, 127, &di) != QAP_OK || di.wide || di.bytevec)
    fail("int16 flows", 20, 0, 0, {});
  if (admit(20, 99, 128, &di) != QAP_OK || !di.wide) fail("D beyond int8", 20, 0, 0, {});
  if (admit(20, 32768, 1, &di) != QAP_OK || !di.wide) fail("F beyond int16", 20, 0, 0, {});
  // B = 52 * 2^40 * 2^19 = 2^64.7: refused; F = 2^40, D = 2^15, n = 2: B = 52 * 2^55 < 2^62
  if (admit(2, (int64_t)1 << 40, 1 << 19, &di) != QAP_EOVERFLOW) fail("bound", 2, 0, 0, {});
  if (admit(2, (int64_t)1 << 40, 1 << 15, &di) != QAP_OK || !di.wide)
    fail("big flows admitted", 2, 0, 0, {});
  if (admit(3, INT64_MIN, 1, &di) != QAP_EOVERFLOW) fail("INT64_MIN", 3, 0, 0, {});
  if (admit(257, 0, 0, &di) != QAP_EUNSUPPORTED) fail("n beyond 256", 257, 0, 0, {});
  // the spreads that decide the byte-vector form and the products form's
  // one-dp2a update (differences of two F entries within int16, of two D
  // entries within int8): one entry lo, the rest hi
  auto spread = [](int n, int64_t flo, int64_t fhi, int64_t dlo, int64_t dhi,
                   qaph::DevInstance* di) {
    std::vector<int64_t> F((size_t)n * n, fhi), D((size_t)n * n, dhi);
    F[1] = flo;
    D[1] = dlo;
    return qaph::inspect_instance(F.data(), D.data(), n, di);
  };
  if (spread(20, 0, 32767, 0, 127, &di) != QAP_OK || di.wide || di.bytevec || !di.diff16)
    fail("F spread 2^15 - 1", 20, 0, 0, {});
  if (spread(20, -1, 32767, 0, 127, &di) != QAP_OK || di.wide || di.diff16)
    fail("F spread 2^15", 20, 0, 0, {});
  if (spread(20, 0, 99, -1, 127, &di) != QAP_OK || di.wide || di.bytevec || di.diff16)
    fail("D spread 128", 20, 0, 0, {});
  if (spread(20, -27, 100, 0, 127, &di) != QAP_OK || !di.bytevec || !di.diff16)
    fail("byte vectors", 20, 0, 0, {});
}

// The search parameters' phase X form: AUTO or DOTS, nothing else.
void check_params() {
  qap_search_params p{};
  p.starts = 1;
  for (int form : {-1, 0, 1, 2}) {
    p.phase_x = form;
    const bool ok = qaph::validate_params(&p) == QAP_OK;
    if (ok != (form == QAP_PHASE_X_AUTO || form == QAP_PHASE_X_DOTS))
      fail("phase_x validation", form, 0, 0, {});
  }
}

int main() {
  if (qapk::row_segments(256, qaph::kLargePlan.maxpt) > qaph::kLargePlan.nt) {
    std::printf("FAIL the large plan does not hold n = 256\n");
    return 1;
  }
  check_admission();
  check_params();
  check_choose_plan();
  check_choose_plan_fit();
  if (fails) {
    std::printf("%d violations\n", fails);
    return 1;
  }
  std::printf("ok\n");
  return 0;
}
