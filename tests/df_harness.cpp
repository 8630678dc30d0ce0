// Host build of the double-float header for tests/test_df_arith.py: reads "op a_hi a_lo b_hi b_lo" lines
// (floats as hex bit patterns), or "split v" / "row nk b d x f_0 q_0 ..." lines (doubles as 64-bit hex
// patterns), and prints the result's two parts as hex bit patterns.
#include <cstdio>
#include <cstring>
#include <cstdint>

#include "../paper_1711_04060_gb300/csrc/pf_df.cuh"

static float fb(uint32_t u) { float f; std::memcpy(&f, &u, 4); return f; }
static uint32_t bf(float f) { uint32_t u; std::memcpy(&u, &f, 4); return u; }

static double db(unsigned long long u) { double v; std::memcpy(&v, &u, 8); return v; }

int main() {
  const pf::Exp2Table T = pf::make_exp2_table();
  char op[16];
  unsigned a, b, c, d;
  while (std::scanf("%15s", op) == 1) {
    // doubles as 64-bit hex patterns: "split v" and "row nk b d x f_0 q_0 ... f_{nk-1} q_{nk-1}"
    if (!std::strcmp(op, "split") || !std::strcmp(op, "row")) {
      unsigned long long w;
      pf::dfl r{0.f, 0.f};
      if (!std::strcmp(op, "split")) {
        if (std::scanf("%llx", &w) != 1) return 1;
        r = pf::df_from_double_bits(db(w));
      } else {
        int nk = 0;
        if (std::scanf("%d", &nk) != 1 || nk < 0 || nk > 6) return 1;
        double v[3], f[6], q[6];
        for (int i = 0; i < 3; ++i) {
          if (std::scanf("%llx", &w) != 1) return 1;
          v[i] = db(w);
        }
        for (int k = 0; k < nk; ++k) {
          if (std::scanf("%llx", &w) != 1) return 1;
          f[k] = db(w);
          if (std::scanf("%llx", &w) != 1) return 1;
          q[k] = db(w);
        }
        r = pf::df_residual_row(v[0], v[1], v[2], f, q, nk);
      }
      std::printf("%08x %08x\n", bf(r.hi), bf(r.lo));
      continue;
    }
    if (std::scanf("%x %x %x %x", &a, &b, &c, &d) != 4) return 1;
    const pf::dfl x{fb(a), fb(b)}, y{fb(c), fb(d)};
    pf::dfl r{0.f, 0.f};
    if (!std::strcmp(op, "exp")) r = pf::df_exp(x, T.hi, T.lo);
    else if (!std::strcmp(op, "add")) r = pf::df_add(x, y);
    else if (!std::strcmp(op, "mul")) r = pf::df_mul(x, y);
    else if (!std::strcmp(op, "addf")) r = pf::df_add_f(x, y.hi);
    else if (!std::strcmp(op, "mulf")) r = pf::df_mul_f(x, y.hi);
    std::printf("%08x %08x\n", bf(r.hi), bf(r.lo));
  }
  return 0;
}
