"""The bit-exact host parity of the library, collected again in the GPU session.

The plan DP, the exact-sum statistics, the landscapes, the decomposition and the
KOL grades are host C++ inside librg.so, rebuilt by the GPU host's own compiler
(an aarch64 build on a Grace host).  The tests of test_abi_host.py prove those
tables and values equal to the oracle's bit for bit; this module re-collects them
with the gpu marker, so that they also run against the build whose numbers a
benchmark on that host reports: full-grid T0*/T1/T2/action/q, leaves, the
tie-heavy seeded cases, surface statistics (including the wide dynamic range),
landscapes, rg_decompose, rg_kol, the pad-only fine-grid plan, FP8 plans, the variant
descriptions and the stream-K schedule's cover."""
import pytest

from test_abi_host import (  # noqa: F401  (re-collected tests and their fixture)
    rg,
    test_decompose_matches_oracle_bit_exact,
    test_fp8_plan_tables_match_oracle,
    test_kol_matches_oracle,
    test_landscapes_match_oracle_bit_exact,
    test_library_exports_every_header_function,
    test_lookup_rounds_up_and_rejects_beyond_grid,
    test_pad_only_plan_on_a_fine_offset_grid_matches_oracle,
    test_plan_leaves_match_oracle_medium_grid,
    test_plan_save_load_roundtrip_and_checksum,
    test_plan_tables_match_oracle_full_grid,
    test_plan_tables_match_oracle_small,
    test_plan_tables_match_oracle_with_many_ties_seeded,
    test_surface_stats_bit_exact_over_a_wide_dynamic_range,
    test_surface_stats_match_oracle_bit_exact,
    test_streamk_geometry_covers_every_k_iteration_once,
    test_surface_stats_non_step_grid,
    test_variant_desc_agrees_with_the_binding,
)

pytestmark = pytest.mark.gpu
