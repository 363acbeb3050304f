"""Host-side checks of the C-ABI library (no GPU needed): it loads, exports every
entry point declared in include/embedjoin.h, its host-only calls answer, and the
Python binding's struct layouts match the header."""
import ctypes as C
import os
import re
import subprocess

import pytest

from conftest import ROOT

HEADER = os.path.join(ROOT, "include", "embedjoin.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1702_00093_gb300 import build
    build.build()
    from paper_1702_00093_gb300 import embedjoin
    return embedjoin.lib()


def declared_functions():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(ej_\w+)\s*\(", src, re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for need in ["ej_embed", "ej_lsh_candidates", "ej_verify", "ej_join", "ej_create", "ej_destroy",
                 "ej_set_test_tables", "ej_sign", "ej_plan"]:
        assert need in names


def test_library_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert len(names) >= 12
    out = subprocess.run(["nm", "-D", "--defined-only", lib._name], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT\s+(\w+)$", out, re.M))
    for nme in names:
        assert nme in exported, nme
        getattr(lib, nme)


def test_binding_lists_every_declared_symbol():
    from paper_1702_00093_gb300 import embedjoin
    assert sorted(embedjoin.EXPORTED) == declared_functions()


def test_status_strings(lib):
    assert lib.ej_status_string(0) == b"ok"
    assert lib.ej_status_string(3) == b"output capacity exceeded"
    assert lib.ej_status_string(99) == b"unknown status"


def test_create_rejects_missing_device(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = C.c_void_p()
    assert lib.ej_create(C.byref(h), 0) != 0
    assert not h.value


def test_struct_layouts_match_header(tmp_path):
    from paper_1702_00093_gb300 import embedjoin as ej
    probe = tmp_path / "probe.c"
    probe.write_text(f'''
#include <stdio.h>
#include <stddef.h>
#include "{HEADER}"
#define F(T, f) printf("%s.%s %zu %zu\\n", #T, #f, offsetof(T, f), sizeof(((T*)0)->f));
int main(void) {{
  printf("ej_params %zu\\n", sizeof(ej_params));
  printf("ej_strings %zu\\n", sizeof(ej_strings));
  printf("ej_plan_info %zu\\n", sizeof(ej_plan_info));
  printf("ej_join_stats %zu\\n", sizeof(ej_join_stats));
  printf("ej_schedule %zu\\n", sizeof(ej_schedule));
  printf("ej_server_config %zu\\n", sizeof(ej_server_config));
  printf("ej_search_result %zu\\n", sizeof(ej_search_result));
  printf("ej_server_stats %zu\\n", sizeof(ej_server_stats));
  F(ej_params, seed) F(ej_params, alphabet) F(ej_params, alphabet_size) F(ej_params, K)
  F(ej_plan_info, embedding_bytes) F(ej_plan_info, key_count)
  F(ej_join_stats, ms_prepare) F(ej_join_stats, ms_total) F(ej_join_stats, ms_pack) F(ej_join_stats, ms_dedup)
  F(ej_schedule, warps_per_subpartition) F(ej_schedule, order) F(ej_schedule, buckets) F(ej_schedule, chain)
  F(ej_tune_entry, schedule) F(ej_tune_entry, back_ms)
  printf("ej_tune_entry %zu\\n", sizeof(ej_tune_entry));
  F(ej_server_config, max_batch_bytes) F(ej_server_config, hbm_reserve) F(ej_server_config, hbm_budget)
  F(ej_search_result, status) F(ej_search_result, matches) F(ej_search_result, queue_ms)
  F(ej_server_stats, deferred) F(ej_server_stats, p99_ms) F(ej_server_stats, device_bytes)
  return 0;
}}''')
    exe = tmp_path / "probe"
    subprocess.check_call(["gcc", "-std=c11", "-o", str(exe), str(probe)])
    got = dict(line.rsplit(" ", 1) if line.count(" ") == 1 else (line.split(" ", 1)[0], line.split(" ", 1)[1])
               for line in subprocess.check_output([str(exe)], text=True).strip().splitlines())
    assert int(got["ej_params"]) == C.sizeof(ej._Params)
    assert int(got["ej_strings"]) == C.sizeof(ej._Strings)
    assert int(got["ej_plan_info"]) == C.sizeof(ej.PlanInfo)
    assert int(got["ej_join_stats"]) == C.sizeof(ej.JoinStats)
    assert int(got["ej_tune_entry"]) == C.sizeof(ej.TuneEntry)
    assert int(got["ej_schedule"]) == C.sizeof(ej._Schedule)
    assert int(got["ej_server_config"]) == C.sizeof(ej.ServerConfig)
    assert int(got["ej_search_result"]) == C.sizeof(ej.SearchResult)
    assert int(got["ej_server_stats"]) == C.sizeof(ej.ServerStats)
    pairs = {"ej_params": ej._Params, "ej_plan_info": ej.PlanInfo, "ej_join_stats": ej.JoinStats,
             "ej_schedule": ej._Schedule, "ej_server_config": ej.ServerConfig,
             "ej_search_result": ej.SearchResult, "ej_server_stats": ej.ServerStats, "ej_tune_entry": ej.TuneEntry}
    for key, val in got.items():
        if "." not in key:
            continue
        sname, field = key.split(".")
        off, size = map(int, val.split())
        assert getattr(pairs[sname], field).offset == off, key
        assert getattr(pairs[sname], field).size == size, key


def test_null_handles_are_rejected_without_a_device(lib):
    # argument checks that need no CUDA call: NULL handles and outputs
    EJ_ERR_INVALID_ARG = 1
    ms = C.c_float(1.0)
    n = C.c_int64(5)
    assert lib.ej_batch_run(None, None) == EJ_ERR_INVALID_ARG
    assert lib.ej_batch_verify_ms(None, C.byref(ms)) == EJ_ERR_INVALID_ARG
    assert lib.ej_batch_result(None, 0, None, 0, C.byref(n), None, None) == EJ_ERR_INVALID_ARG
    assert lib.ej_batch_kernel_count(None) == 0
    assert lib.ej_index_size(None) == 0
    assert lib.ej_server_submit(None, None, 0, 1) == -EJ_ERR_INVALID_ARG
    assert lib.ej_server_submit(None, None, 0, -1) == -EJ_ERR_INVALID_ARG
    n32 = C.c_int32(3)
    assert lib.ej_server_poll(None, None, 0, C.byref(n32), 0) == EJ_ERR_INVALID_ARG
    assert lib.ej_server_release(None, 0) == EJ_ERR_INVALID_ARG
    assert lib.ej_server_get_stats(None, None) == EJ_ERR_INVALID_ARG
    assert lib.ej_server_reset_stats(None) == EJ_ERR_INVALID_ARG
    lib.ej_batch_destroy(None)
    lib.ej_index_destroy(None)
    lib.ej_server_destroy(None)
