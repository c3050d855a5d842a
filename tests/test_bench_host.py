"""Host logic of bench.py (no GPU): the kernel form named for each plan
variant id that fstat_get_plan can report (include/fstat.h; the far-field
table of csrc/api.cu, reported as 100 + its index)."""
import bench


def test_variant_ids_name_their_form():
    assert all(bench.algo_of(v) == "direct" for v in range(0, 100))
    # far-field form: rounds staging (100-106), TMA ring (107-111), ring with coverage (117),
    # blocks of 4 sky points (132)
    assert all(bench.algo_of(v) == "farpoly" for v in list(range(100, 112)) + [117, 132])
    # sinc ring: 10 and 8 compute warps (112-115), coverage (116), L = 1 (118-119),
    # 4 and 2 compute warps (129-130), blocks of 4 sky points (131, 133, 134)
    assert all(bench.algo_of(v) == "sincpoly" for v in [112, 113, 114, 115, 116, 118, 119, 129, 130, 131, 133, 134])
    assert all(bench.algo_of(v) == "sincrows" for v in range(120, 127))
    assert all(bench.algo_of(v) == "sincpairs" for v in (127, 128))
    # every form has a kernel name and source list for the roofline and counters keys
    for form in ("direct", "farpoly", "sincpoly", "sincrows", "sincpairs"):
        assert form in bench.KERNEL_NAMES and form in bench.KERNEL_SOURCES
