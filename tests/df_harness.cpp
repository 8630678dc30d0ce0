// Host build of the double-float header for tests/test_df_arith.py: reads "op a_hi a_lo b_hi b_lo" lines
// (floats as hex bit patterns) and prints the result's two parts as hex bit patterns.
#include <cstdio>
#include <cstring>
#include <cstdint>

#include "../paper_1711_04060_gb300/csrc/pf_df.cuh"

static float fb(uint32_t u) { float f; std::memcpy(&f, &u, 4); return f; }
static uint32_t bf(float f) { uint32_t u; std::memcpy(&u, &f, 4); return u; }

int main() {
  const pf::Exp2Table T = pf::make_exp2_table();
  char op[16];
  unsigned a, b, c, d;
  while (std::scanf("%15s %x %x %x %x", op, &a, &b, &c, &d) == 5) {
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
