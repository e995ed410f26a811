"""Host-side pieces of bench.py: every kernel path de_get_plan can report
has a name and a launch count."""
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_every_kernel_path_is_named(bench):
    # include/de.h, de_get_plan: paths 0 (FP64 per generation), 1 (split,
    # three kernels), 2 (split, persistent cluster), 3 (FP64, cooperative),
    # 4 (split, persistent with CTA-local products)
    assert sorted(bench.KERNEL_PATH_NAMES) == [0, 1, 2, 3, 4, 5]


@pytest.mark.parametrize("path,expected", [(0, 3 + 3000), (1, 3 + 3 * 3000), (2, 3 + 2), (3, 3 + 1), (4, 3 + 2), (5, 3 + 1)])
def test_launches_per_step(bench, path, expected):
    assert bench.launches_per_step({"kernel_path": path, "cluster_size": 0}, 3000) == expected
