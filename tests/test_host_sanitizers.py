"""The library's host code under the compiler's sanitizers, without a GPU.

The C++ check programs of the other host tests (the factorization, the
operator assembly, the solve schedules and their release protocol replayed by
racing threads, the device decomposition's plan run on the CPU, the top
inverse's plan, the state packing, the constraint split) are built again with
AddressSanitizer and UndefinedBehaviorSanitizer, and the threaded ones that run
in seconds with ThreadSanitizer, and must finish with their usual "ok" and no
sanitizer report: no out-of-bounds access, use after free, leak, undefined
arithmetic or data race in the host code they exercise."""
import concurrent.futures as cf
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2107_05200_gb300", "csrc")

CHECKS = {
    "constraint_check": ["ffa_constraint_host.cpp"],
    "state_check": ["ffa_state.cpp"],
    "operator_check": ["ffa_operator_host.cpp", "ffa_factor.cpp"],
    "topinv_check": ["ffa_factor.cpp", "ffa_topinv_plan.cpp"],
    "schedule_check": ["ffa_factor.cpp", "ffa_schedule.cpp"],
    "devfactor_check": ["ffa_devfactor_plan.cpp", "ffa_factor.cpp", "ffa_operator_host.cpp"],
    "factor_check": ["ffa_factor.cpp"],
}
THREAD_CHECKS = ["operator_check", "schedule_check"]
FLAGS = {"address,undefined": ["-fsanitize=address,undefined", "-fno-sanitize-recover=undefined"],
         "thread": ["-fsanitize=thread"]}


def _build_and_run(gxx, tmp, name, kind):
    exe = os.path.join(tmp, f"{name}_{kind.replace(',', '_')}")
    srcs = [os.path.join(ROOT, "tests", name + ".cpp")] + [os.path.join(CSRC, s) for s in CHECKS[name]]
    subprocess.run([gxx, "-O1", "-g", "-std=c++17", "-pthread", "-fno-omit-frame-pointer", *FLAGS[kind], "-o", exe,
                    *srcs], check=True, capture_output=True, timeout=900)
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1", UBSAN_OPTIONS="print_stacktrace=1",
               TSAN_OPTIONS="halt_on_error=1")
    r = subprocess.run([exe], capture_output=True, text=True, timeout=900, env=env)
    return name, kind, r


def test_host_checks_are_clean_under_the_sanitizers(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no g++")
    probe = subprocess.run([gxx, "-fsanitize=address,undefined", "-x", "c++", "-", "-o", str(tmp_path / "probe")],
                           input="int main() { return 0; }\n", capture_output=True, text=True)
    if probe.returncode != 0:
        pytest.skip("the compiler has no sanitizer runtime")
    jobs = [(n, "address,undefined") for n in CHECKS] + [(n, "thread") for n in THREAD_CHECKS]
    with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 1)) as ex:
        results = list(ex.map(lambda j: _build_and_run(gxx, str(tmp_path), *j), jobs))
    for name, kind, r in results:
        out = r.stdout + r.stderr
        if kind == "thread" and "unexpected memory mapping" in out:
            continue   # this kernel's address-space layout keeps ThreadSanitizer from starting
        # devfactor_check prints one line per plan before its verdict, the others only the verdict
        verdict = r.stdout.strip().splitlines()[-1] if r.stdout.strip() else ""
        assert r.returncode == 0 and verdict.startswith("ok"), (name, kind, out[-3000:])
        for marker in ("ERROR: AddressSanitizer", "ERROR: LeakSanitizer", "runtime error:",
                       "WARNING: ThreadSanitizer"):
            assert marker not in out, (name, kind, out[-3000:])
