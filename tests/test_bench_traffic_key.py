"""bench.py keys the stored DRAM traffic of a Lanczos step (profiles/) to the
step's own kernel source: an edit elsewhere in k_lanczos.cu keeps the key, an
edit to the update kernel or to the step's other sources changes it, and a
lost region marker falls back to hashing the whole file (the stored traffic is
then not used)."""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1912_02949_gb300", "csrc")


def _reader(edit=None):
    def read(name):
        text = open(os.path.join(CSRC, name), encoding="utf-8").read()
        return edit(name, text) if edit else text
    return read


def test_key_covers_the_update_kernel_only():
    lz = open(os.path.join(CSRC, "k_lanczos.cu"), encoding="utf-8").read()
    region = bench.step_source(lz)
    assert "k_lanczos_update(KP<V> p, int i)" in region and "launch_lanczos_update" in region
    assert "k_ritz" not in region and "k_tridiag(KP<V> p" not in region and "k_dual_start" not in region


def test_key_ignores_other_kernels_and_follows_the_step():
    lz = open(os.path.join(CSRC, "k_lanczos.cu"), encoding="utf-8").read()
    assert "constexpr int EPT = W / CF;" in lz                       # in k_ritz: the edits below are real
    assert "constexpr int UN = 2;              // 16-byte groups" in bench.step_source(lz)
    base = bench.kernel_source_sha(_reader())
    ritz_edit = bench.kernel_source_sha(_reader(
        lambda n, t: t.replace("constexpr int EPT = W / CF;", "constexpr int EPT = (W / CF);") if n == "k_lanczos.cu" else t))
    assert ritz_edit == base
    upd_edit = bench.kernel_source_sha(_reader(
        lambda n, t: t.replace("constexpr int UN = 2;              // 16-byte groups", "constexpr int UN = 4;              // 16-byte groups")
        if n == "k_lanczos.cu" else t))
    assert upd_edit != base
    tiled_edit = bench.kernel_source_sha(_reader(lambda n, t: t + "\n" if n == "k_tiled.cu" else t))
    assert tiled_edit != base


def test_lost_marker_hashes_the_whole_file():
    lz = open(os.path.join(CSRC, "k_lanczos.cu"), encoding="utf-8").read()
    broken = lz.replace(bench.STEP_REGIONS[0][0], "// (marker removed)")
    assert bench.step_source(broken) == broken
