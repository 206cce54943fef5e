// Host-only check of the shared-memory layouts of the pipeline kernels for
// every grid size (16 .. 4096) and both precisions: each kernel's dynamic
// shared memory stays within the per-CTA limit, every region that an
// asynchronous copy (bulk copy or cp.async) writes starts on a 16-byte
// boundary and holds what is copied into it, the mbarrier is 8-byte aligned,
// and the prefetching row passes keep the CTAs per SM their registers allow.
// Prints "OK" or the failing checks; exit status 0 on success.
#include <cstdio>

#include "kernels.cuh"
#include "standard.cuh"

static int failures = 0;
static void expect(bool c, const char* what, int log2n, int fp32) {
  if (!c) {
    std::printf("FAIL log2n=%d %s: %s\n", log2n, fp32 ? "fp32" : "fp64", what);
    ++failures;
  }
}

constexpr size_t kMaxSmem = 232448;   // dynamic shared memory per CTA
constexpr size_t kSmSmem = 233472;    // per SM, 1 KB reserved per CTA

template <typename R, int L>
void check() {
  using G = dsnu::Geo<R, L>;
  using S = dsnu::GeoStd<R, L>;
  constexpr int N = G::N;
  constexpr size_t C = sizeof(dsnu::cpx<R>);
  const int f = sizeof(R) == 4;
  // sizes
  expect(G::smem_row_fwd <= kMaxSmem, "row_fwd shared memory", L, f);
  expect(G::smem_row_inv <= kMaxSmem, "row_inv shared memory", L, f);
  expect(G::smem_row_inv_limit <= kMaxSmem, "row_inv limit", L, f);
  expect(G::smem_col <= kMaxSmem, "band passes shared memory", L, f);
  expect(G::smem_col_main <= kMaxSmem, "col_main shared memory", L, f);
  expect(S::smem_rowf <= kMaxSmem && S::smem_rowi <= kMaxSmem && S::smem <= kMaxSmem, "standard passes", L, f);
  // forward row pass: landing rows of rho after the stage table, buffers and half twiddle table
  if (G::ROW_PF) {
    const size_t land = (G::STWCP + 2 * G::RB_F * G::RS + N / 2) * C;
    expect(land % 16 == 0, "row_fwd landing alignment", L, f);
    expect((G::LS * 8) % 16 == 0, "row_fwd landing row stride", L, f);
    const size_t bar = land + size_t(G::RB_F) * G::LS * 8;
    expect(bar % 8 == 0 && bar + 8 <= G::smem_row_fwd, "row_fwd mbarrier", L, f);
    expect(size_t(G::MINB_F0) * (G::smem_row_fwd + 1024) <= kSmSmem, "row_fwd CTAs per SM", L, f);
    expect((size_t(N) * 8) % 16 == 0, "row_fwd bulk copy size", L, f);
  }
  // inverse row pass: landing of the row pair's segments, then the band values
  if (G::ROWI_PF) {
    const size_t land = (G::STWCP + 2 * G::RB_I * G::RS + N / 2) * C;
    expect(land % 16 == 0, "row_inv landing alignment", L, f);
    expect(land + size_t(2 * (N + 1)) * C <= G::smem_row_inv, "row_inv landing size", L, f);
    expect((land + size_t(2 * (N + 1)) * C) % 16 == 0, "row_inv band landing alignment", L, f);
    expect(size_t(G::MINB_I0) * (G::smem_row_inv + 1024) <= kSmSmem, "row_inv CTAs per SM", L, f);
    expect(dsnu::Tile<R>::TR * C == 32, "row tiles of 32 bytes", L, f);
  }
  // column pass: the two multiplier-row buffers after the twiddle table
  if (G::COL_TAB) {
    const size_t mrow = (G::STWP + 2 * G::CC * G::FB + N) * C;
    expect(mrow % 16 == 0, "col_main multiplier rows alignment", L, f);
    expect((G::LDM * 4) % 16 == 0, "col_main multiplier row stride", L, f);
    expect(mrow + size_t(2 * G::CC * G::LDM) * 4 <= G::smem_col_main, "col_main multiplier rows size", L, f);
  }
  // the FFT buffers themselves start 16-byte aligned
  expect((G::STWP * C) % 16 == 0 && (G::STWCP * C) % 16 == 0 && (G::RS * C) % 16 == 0, "buffer alignment", L, f);
  // standard solver landings
  if (S::PF) {
    const size_t landf = (S::STWCP + S::PER * S::FB) * C;
    expect(landf % 16 == 0, "standard row_fwd landing alignment", L, f);
    expect(landf + size_t(2 * S::PER) * N * 8 + 8 <= S::smem_rowf, "standard row_fwd landing size", L, f);
    expect(S::smem_rowi >= landf + size_t(S::PER) * (N / 2 + 1) * 16, "standard row_inv landing size", L, f);
  }
}

template <typename R, int L>
void all() {
  check<R, L>();
  if constexpr (L < 12) all<R, L + 1>();
}

int main() {
  all<float, 4>();
  all<double, 4>();
  if (failures == 0) std::printf("OK\n");
  return failures == 0 ? 0 : 1;
}
