// Host-side check of the shared-memory layout of the TMA-staged z pass (compiled by
// tests/test_zw_layout.py; only compile-time constants are read, nothing runs on a GPU).
#include <cstdio>
#include "passes.cuh"
using namespace lsgpu;

static int failures = 0;
#define REQUIRE(cond, L)                                               \
  do {                                                                 \
    if (!(cond)) {                                                     \
      printf("L=%d: %s fails\n", L, #cond);                            \
      ++failures;                                                      \
    }                                                                  \
  } while (0)

template <int L, bool ALT = false>
void check() {
  using W = ZW<L, ALT>;
  if (!W::ok) return;
  // static shared memory of the kernel: the active-view list, the warp sums and the abort flag
  constexpr size_t static_smem = kMaxLaunchSlots * sizeof(int) + 32 * sizeof(int) + 16;
  constexpr size_t sm_capacity = 228 * 1024, per_cta_max = 227 * 1024, reserved_per_cta = 1024;
  // every region starts on a 16-byte boundary (TMA tiles, 16-byte exchange and twiddle loads, mbarriers)
  REQUIRE(W::stage_bytes % 1024 == 0, L);
  REQUIRE(W::off_g % 16 == 0 && W::off_x % 16 == 0, L);
  REQUIRE(W::off_twa % 16 == 0 && W::off_twb % 16 == 0 && W::off_bar % 16 == 0, L);
  // the regions do not overlap, except the exchange area overlaying the Green tile when the Green
  // values live in registers
  REQUIRE(W::off_g >= (size_t)W::NS * W::stage_bytes, L);
  REQUIRE(W::off_twa >= W::off_x + W::x_bytes, L);
  REQUIRE(W::GREG || W::off_x >= W::off_g + W::g_bytes, L);   // Green tile only without GREG
  REQUIRE(W::off_twb >= W::off_twa + (size_t)W::R2 * W::TWA * sizeof(float2), L);
  REQUIRE(W::off_bar >= W::off_twb + (size_t)W::R1 * W::TWB * sizeof(float2), L);
  REQUIRE(W::NBAR == 2 * W::NS + 1 && W::smem >= W::off_bar + W::NBAR * sizeof(uint64_t) + 1023, L);
  // exchange rows: R1 rows of R2 + 2 and R2 rows of R1 + 2 entries fit a column's pitch, and the
  // rows and pitch are even so that 16-byte reads stay aligned
  REQUIRE(W::R1 * (W::R2 + 2) <= W::XP && W::R2 * (W::R1 + 2) <= W::XP, L);
  REQUIRE(W::XP % 2 == 0 && W::R1 % 2 == 0 && W::R2 % 2 == 0, L);
  REQUIRE((size_t)W::P * W::XP * sizeof(float2) <= W::x_bytes, L);
  // twiddle rows read as float4 pairs
  REQUIRE(W::TWA % 2 == 0 && W::TWB % 2 == 0, L);
  // the resident CTAs the launch bounds ask for fit one SM
  REQUIRE(W::smem <= per_cta_max, L);
  REQUIRE((size_t)W::MINB * (W::smem + static_smem + reserved_per_cta) <= sm_capacity, L);
  printf("L=%3d split %2dx%-2d NS=%d smem %6zu B x %d CTAs/SM\n", L, W::R1, W::R2, W::NS, W::smem, W::MINB);
}

// The column-group z pass (k_zg): the same layout rules, plus the thread mapping of its groups.
template <int L>
void check_groups() {
  using W = ZG<L>;
  if (!W::ok) return;
  constexpr size_t static_smem = kMaxLaunchSlots * sizeof(int) + 32 * sizeof(int) + 16;
  constexpr size_t sm_capacity = 228 * 1024, per_cta_max = 227 * 1024, reserved_per_cta = 1024;
  REQUIRE(W::CG * W::T == 32 * W::WG && W::NGRP * W::CG == W::P && W::R2 % W::T == 0 && W::R1 == W::T, L);
  REQUIRE(W::stage_bytes % 1024 == 0, L);
  REQUIRE(W::off_x % 16 == 0 && W::off_twa % 16 == 0 && W::off_twb % 16 == 0 && W::off_bar % 16 == 0, L);
  REQUIRE(W::off_x >= (size_t)W::NS * W::stage_bytes, L);
  REQUIRE(W::off_twa >= W::off_x + W::x_bytes && W::off_g == W::off_x && W::off_twa >= W::off_g + W::g_bytes, L);
  REQUIRE(W::GR % 16 == 8 && W::GR >= W::P, L);
  REQUIRE(W::off_twb >= W::off_twa + (size_t)W::R2 * W::TWA * sizeof(float2), L);
  REQUIRE(W::off_bar >= W::off_twb + (size_t)W::R1 * W::TWB * sizeof(float2), L);
  REQUIRE(W::NBAR == 2 * W::NS + 1 && W::smem >= W::off_bar + W::NBAR * sizeof(uint64_t) + 1023, L);
  REQUIRE(W::R1 * W::RA <= W::XP && W::R2 * W::RB <= W::XP, L);
  REQUIRE(W::XP % 16 == 2 && W::RA % 2 == 0 && W::RB % 2 == 0, L);
  REQUIRE((size_t)W::P * W::XP * sizeof(float2) <= W::x_bytes, L);
  REQUIRE(W::smem <= per_cta_max, L);
  REQUIRE((size_t)W::MINB * (W::smem + static_smem + reserved_per_cta) <= sm_capacity, L);
  // every row read from the stage buffer and every output row lies in the tile
  REQUIRE(W::R2 * (W::R1 / 2 - 1) + (W::R2 - 1) < W::NZ, L);
  printf("L=%3d groups %dx%d (T=%d, S1=%d) NS=%d smem %6zu B x %d CTAs/SM\n", L, W::R1, W::R2, W::T, W::S1, W::NS,
         W::smem, W::MINB);
}

// The dynamically scheduled z pass (k_zwd): view buffers, the swizzled Green tile (a TMA destination:
// 1024-byte aligned), exchange, twiddles and barriers, for the resident CTAs its launch bounds ask for.
template <int L>
void check_dyn() {
  using W = ZWD<L>;
  if (!W::ok) return;
  constexpr size_t static_smem = kMaxLaunchSlots * sizeof(int) + 32 * sizeof(int) + 16 + W::NS * sizeof(int);
  static_assert(static_smem == W::static_smem, "static shared memory of k_zwd");
  constexpr size_t sm_capacity = 228 * 1024, per_cta_max = 227 * 1024, reserved_per_cta = 1024;
  REQUIRE(W::stage_bytes % 1024 == 0 && W::off_g % 1024 == 0, L);
  REQUIRE(W::off_g >= (size_t)W::NS * W::stage_bytes && W::off_x >= W::off_g + W::gtile_bytes, L);
  REQUIRE(W::off_x % 16 == 0 && W::off_twa % 16 == 0 && W::off_twb % 16 == 0 && W::off_bar % 16 == 0, L);
  REQUIRE(W::off_twa >= W::off_x + W::x_bytes, L);
  REQUIRE(W::off_twb >= W::off_twa + (size_t)W::R2 * W::TWA * sizeof(float2), L);
  REQUIRE(W::off_bar >= W::off_twb + (size_t)W::R1 * W::TWB * sizeof(float2), L);
  REQUIRE(W::NBAR == 2 * W::NS + 3 && W::smem >= W::off_bar + W::NBAR * sizeof(uint64_t) + 1023, L);
  REQUIRE(W::NZ + 1 <= 256 && W::gtile_bytes == (size_t)(W::NZ + 1) * 128, L);   // one TMA box of Green rows
  REQUIRE(W::smem <= per_cta_max, L);
  REQUIRE((size_t)W::MINB * (W::smem + static_smem + reserved_per_cta) <= sm_capacity, L);
  printf("L=%3d dynamic split %2dx%-2d NS=%d smem %6zu B x %d CTAs/SM\n", L, W::R1, W::R2, W::NS, W::smem, W::MINB);
}

// The z-pass form untuned plans run for a length (ZAuto) exists for it: the round-robin persistent
// form needs register-resident Green values, the dynamic form its own layout; lengths without the
// TMA-staged pass (the bead lengths run the column-group pass) may name any form.
template <int L>
void check_auto() {
  constexpr int forms[2] = {ZAuto<L>::small, ZAuto<L>::large};
  for (int f : forms) {
    REQUIRE(f >= 0 && f <= 2, L);
    if (ZW<L>::ok) {
      if (f == 1) REQUIRE(ZW<L>::GREG, L);
      if (f == 2) REQUIRE(ZWD<L>::ok, L);
    }
  }
}

int main() {
  check_groups<144>(); check_groups<288>();
  check<16>(); check<24>(); check<32>(); check<48>(); check<64>(); check<96>(); check<128>();
  check<144>(); check<192>(); check<256>(); check<288>(); check<384>();
  // the second splits the autotuner can choose
  check<16, true>(); check<24, true>(); check<32, true>(); check<48, true>(); check<64, true>(); check<96, true>();
  check<128, true>(); check<192, true>(); check<256, true>(); check<384, true>();
  check_dyn<16>(); check_dyn<32>(); check_dyn<48>(); check_dyn<64>(); check_dyn<96>(); check_dyn<128>();
  check_dyn<192>(); check_dyn<256>(); check_dyn<384>();
  check_auto<16>(); check_auto<24>(); check_auto<32>(); check_auto<48>(); check_auto<64>(); check_auto<96>();
  check_auto<128>(); check_auto<144>(); check_auto<192>(); check_auto<256>(); check_auto<288>(); check_auto<384>();
  printf(failures ? "FAIL\n" : "OK\n");
  return failures ? 1 : 0;
}
