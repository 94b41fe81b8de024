"""The committed ncu counters are keyed by the code of the stage-kernel
sources: a comment or spacing edit must keep the key, any code change must
drop it (CPU)."""
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
