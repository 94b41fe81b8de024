"""The committed ncu counters are keyed by the code of the stage-kernel
sources and their compile flags: a comment or spacing edit must keep the
key, any code or flag change must drop it (CPU)."""
import bench


def test_code_only_ignores_comments_and_spacing():
    a = "int f(int x) {  // the answer\n    return x + 1; /* add\n one */\n}\n"
    b = "int f(int x) {\n  return x + 1;\n}   // edited comment\n"
    assert bench._code_only(a) == bench._code_only(b)


def test_code_only_sees_code_changes():
    a = "float g(float x) { return 0.5f * x; }"
    b = "float g(float x) { return 0.25f * x; }"
    assert bench._code_only(a) != bench._code_only(b)


def test_committed_counters_match_the_current_sources():
    # the committed summary was taken on the current stage-kernel code
    assert bench.committed_traffic("stage2") is not None
    assert bench.committed_counter("warp_instructions", "stage2") is not None


def test_flags_are_part_of_the_key(monkeypatch):
    from paper_1912_02457_gb300 import build
    k0 = bench.kernel_source_hash()
    flags = dict(build.FILE_FLAGS)
    flags["swe_stage_fast.cu"] = flags["swe_stage_fast.cu"] + ["-DSOMETHING"]
    monkeypatch.setattr(build, "FILE_FLAGS", flags)
    assert bench.kernel_source_hash() != k0
