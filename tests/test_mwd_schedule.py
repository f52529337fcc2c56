"""CPU check of the blocked kernel's schedule (bounds, levels read, one-barrier-per-step races)."""
import pytest

from mwd_schedule_model import simulate

CASES = [
    # R, second order, nx, ny, nz, T, dw, nf, C
    (1, False, 37, 19, 7, 9, 4, 1, 1),
    (1, False, 70, 23, 6, 5, 8, 2, 2),
    (1, False, 70, 17, 5, 8, 16, 1, 4),
    (1, False, 40, 13, 6, 7, 6, 3, 2),
    (1, False, 3, 2, 5, 5, 2, 1, 1),
    (1, False, 65, 9, 4, 11, 4, 4, 4),
    (4, True, 70, 29, 12, 5, 8, 1, 1),
    (4, True, 46, 35, 11, 9, 16, 2, 2),
    (4, True, 44, 30, 10, 6, 24, 1, 4),
    (4, True, 70, 29, 9, 7, 16, 1, 8),
    (1, False, 70, 12, 5, 6, 4, 1, 16),
    (4, True, 5, 7, 3, 5, 8, 1, 1),
]


MODES = [(c, m) for c in CASES for m in ("element", "vec_f32", "bulk_f32")] + \
        [(c, m) for c in CASES[1::2] for m in ("vec_f64", "bulk_f64")]


@pytest.mark.parametrize("case", [c for c in CASES if c[0] == 1])
def test_schedule_model_box_stencil(case):
    """The 27-point box stencil's diagonal reads (Sect. 8.4: the tiles already cover edge and corner
    dependencies) find level t in every ring slot and halo column they touch."""
    for a16 in (4, 2):
        assert simulate(*case, vec=True, a16=a16, box=True)


@pytest.mark.parametrize("case,mode", MODES)
def test_schedule_model(case, mode):
    if mode == "element":
        assert simulate(*case)
    else:
        assert simulate(*case, vec=True, bulk=mode.startswith("bulk"), a16=4 if mode.endswith("f32") else 2)
