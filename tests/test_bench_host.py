"""Host-side pieces of bench.py that need no GPU: the cycle options' labels and
sweep counts, the algorithmic-byte model, and the oracle baseline of the
random-game batch."""
import bench
import synth


def test_cycle_sweeps_and_labels():
    assert bench.cycle_sweeps({"nu1": 1, "nu2": 2}) == (3, 3)
    assert bench.cycle_sweeps({"nu1": 1, "nu2": 2, "nu2_coarse": 1}) == (3, 2)
    assert bench.cycle_sweeps({"nu1": 2, "nu2": 1, "nu1_coarse": 0, "nu2_coarse": 2}) == (3, 2)
    assert bench.cycle_label({"nu1": 1, "nu2": 2}) == "V(1,2)"
    assert bench.cycle_label({"nu1": 1, "nu2": 2, "nu2_coarse": 1}) == "V(1,2), coarse levels (1,1)"


def test_byte_model_grows_with_sweeps():
    for prec in ("fp64", "mixed", "mixed_bf16"):
        b2, b3 = bench.mg_bytes_per_state(prec, 2), bench.mg_bytes_per_state(prec, 3)
        assert b3["cycle"] > b2["cycle"] and b3["check"] == b2["check"]
        # fewer coarse sweeps move fewer bytes, by the coarse levels' share only
        bc = bench.mg_bytes_per_state(prec, 3, 2)
        assert b2["cycle"] < bc["cycle"] < b3["cycle"]
    # bfloat16 weights move fewer bytes than float32 ones
    assert bench.mg_bytes_per_state("mixed_bf16")["cycle"] < bench.mg_bytes_per_state("mixed")["cycle"]
    # launches x check + cycles x (cycle + check)
    b = bench.mg_bytes_per_state("mixed", 3)
    assert bench.mg_cycle_bytes(10, "mixed", 2, 5, 3) == 10 * (2 * b["check"] + 5 * (b["cycle"] + b["check"]))


def test_oracle_batch_baseline_runs_on_the_host():
    sizes = synth.batch_game_sizes(64, 4, nmin=64, nmax=128)
    games_per_s, cores, cpu_s = bench.oracle_batch_sample(sizes, 4, games=4, workers=2)
    assert games_per_s > 0 and cores == 2 and cpu_s > 0
