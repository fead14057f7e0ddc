"""The algorithmic flop tallies behind the bench's rooflines (no GPU).

bench.FLOP_TALLY itemises one retarded pair evaluation (point, charge, time) of the plain per-charge
method: the retarded time as the root of a quadratic on one linear history segment, linear
interpolation of position, velocity and acceleration there, and Griffiths' E, B, phi, A added to
the sums (an add, multiply, divide, square root or reciprocal square root 1 flop, a dot product of
3-vectors 5, a fused multiply-add 2).  bench.DRIVE_FLOP_TALLY is the same evaluation for one
charge's share of an oscillator's driving field: E alone, projected on the receiver's axis.
"""
import bench


def _total(t):
    return sum(sum(v.values()) for v in t.values())


def test_field_tally():
    t = bench.FLOP_TALLY
    assert sum(t["retarded time (quadratic on one segment)"].values()) == 34
    assert sum(t["interpolation at the root"].values()) == 27
    assert sum(t["Lienard-Wiechert fields (Griffiths)"].values()) == 85
    assert _total(t) == bench.FLOPS_PER_PAIR == 146


def test_drive_tally_is_the_field_tally_for_p_dot_E():
    f = bench.FLOP_TALLY["Lienard-Wiechert fields (Griffiths)"]
    accumulations = f["E +="] + f["B += n x E / c"] + f["phi += k q c / (R u)"] + f["A += (phi / c^2) v"]
    projection = sum(bench.DRIVE_FLOP_TALLY["projection"].values())
    assert accumulations == 27 and projection == 6
    assert bench.DRIVE_FLOPS_PER_PAIR == bench.FLOPS_PER_PAIR - accumulations + projection == 125
    # the retarded time and the interpolation are those of the field evaluation
    for k in ("retarded time (quadratic on one segment)", "interpolation at the root"):
        assert bench.DRIVE_FLOP_TALLY[k] == bench.FLOP_TALLY[k]
