"""The C ABI from a C program (no Python between the caller and the
library): a C11 client compiled against include/tc.h and linked with
libtc_gb300.so reads an edge-list file and runs the server's scheduler in its
fake mode.  Host work only: runs without a GPU."""
import os
import shutil
import subprocess

import pytest

import paper_1708_06866_gb300 as tc
from conftest import ROOT

CLIENT = r"""
#include <stdio.h>
#include <string.h>
#include "tc.h"

int main(int argc, char** argv) {
    int32_t src[16], dst[16];
    int64_t m = 0;
    int32_t n = 0;
    int rc = tc_read_edges(argv[1], 0, NULL, NULL, 0, &m, &n);
    if (rc != TC_OK || m != 5) { printf("count rc=%d m=%lld\n", rc, (long long)m); return 1; }
    rc = tc_read_edges(argv[1], 0, src, dst, 16, &m, &n);
    if (rc != TC_OK) { printf("read rc=%d %s\n", rc, tc_last_error()); return 1; }
    printf("edges %lld n %d first %d-%d last %d-%d\n", (long long)m, n, src[0], dst[0],
           src[m - 1], dst[m - 1]);
    if (tc_read_edges("/nonexistent/x.tsv", 0, NULL, NULL, 0, &m, &n) != TC_EINVAL) return 1;
    printf("missing file: %s\n", tc_strerror(TC_EINVAL));

    tc_debug_server_fake(1);
    tc_graph_source g[2];
    memset(g, 0, sizeof(g));
    for (int i = 0; i < 2; ++i) { g[i].src = src; g[i].dst = dst; g[i].m_in = 5; g[i].n = n; }
    tc_server* s = NULL;
    rc = tc_server_create(g, 2, (int64_t)1 << 30, 40, 3, &s);
    if (rc != TC_OK) { printf("create rc=%d %s\n", rc, tc_last_error()); return 1; }
    tc_request r[4];
    tc_response out[4];
    memset(r, 0, sizeof(r));
    for (int i = 0; i < 4; ++i) {
        r[i].graph = i & 1;
        r[i].kind = i < 2 ? TC_REQ_COUNT : TC_REQ_KTRUSS;
        r[i].k = 3 + i;
    }
    double wall = 0;
    rc = tc_server_run(s, r, 4, 0, 0, out, &wall);
    if (rc != TC_OK) { printf("run rc=%d %s\n", rc, tc_last_error()); return 1; }
    for (int i = 0; i < 4; ++i) printf("result %d %lld\n", i, (long long)out[i].result);
    tc_server_stats st;
    tc_server_get_stats(s, &st);
    printf("builds %lld violations %lld\n", (long long)st.builds, (long long)st.violations);
    tc_server_destroy(s);
    tc_debug_server_fake(0);
    return 0;
}
"""


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_c_client(tmp_path):
    lib = tc.library_path()
    tc.load_library()                       # builds the library if needed
    (tmp_path / "client.c").write_text(CLIENT)
    exe = tmp_path / "client"
    subprocess.run(["gcc", "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                    str(tmp_path / "client.c"), lib, f"-Wl,-rpath,{os.path.dirname(lib)}",
                    "-o", str(exe)], check=True)
    edges = tmp_path / "g.tsv"
    edges.write_text("1\t2\t1\n2\t3\t1\n3\t1\t1\n3\t4\t1\n# comment\n4\t5\t1\n")
    out = subprocess.run([str(exe), str(edges)], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0, out.stdout + out.stderr
    lines = out.stdout.splitlines()
    assert lines[0] == "edges 5 n 5 first 0-1 last 3-4"
    assert lines[1].startswith("missing file:")
    assert lines[2:6] == ["result 0 0", "result 1 1000", "result 2 5", "result 3 1006"]
    assert lines[6] == "builds 2 violations 0"
