"""The C-ABI boundary without a GPU: the library builds for sm_103a, loads with
every symbol bound at load time, exports every function include/*.h declares,
and the Python binding declares the same set.  The oracle library builds and
loads too.  No compute call is made."""
import ctypes
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b(dwf_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


def test_header_declares_the_api():
    names = declared_functions()
    for n in ("dwf_create", "dwf_apply", "dwf_cg", "dwf_mspcg", "dwf_batch_mspcg",
              "dwf_set_reduced_ls", "dwf_destroy", "dwf_last_error"):
        assert n in names
    assert len(names) >= 30


def test_library_loads_and_exports_every_declared_function():
    from paper_2104_05615_gb300 import build
    lib_path = build.build()
    # RTLD_NOW: an unresolved reference fails here, not at its first call
    lib = ctypes.CDLL(lib_path, mode=ctypes.RTLD_LOCAL | os.RTLD_NOW)
    missing = [n for n in sorted(declared_functions()) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_declares_every_function():
    from paper_2104_05615_gb300 import binding
    src = open(binding.__file__).read()
    missing = [n for n in sorted(declared_functions()) if f'"{n}"' not in src]
    assert not missing, missing


def test_oracle_library_builds_and_loads():
    import oracle
    path = oracle.build()
    ctypes.CDLL(path, mode=ctypes.RTLD_LOCAL | os.RTLD_NOW)


C_CLIENT = r"""
#include <stdio.h>
#include <string.h>
#include "dwf.h"

static int fail(const char *what) { fprintf(stderr, "%s\n", what); return 1; }

int main(void)
{
    dwf_solver_params p;
    dwf_handle *h = NULL;
    double g[2 * 4 * 9 * 2] = {0};
    const int odd[4] = {3, 4, 4, 4}, sub[4] = {4, 4, 4, 4};
    double t = 0.0;
    dwf_default_params(&p);
    if (p.tol != 1e-10 || p.inner_iters != 6 || p.inner_prec != DWF_F16 || p.outer_prec != DWF_F32)
        return fail("default parameters");
    if (!dwf_status_string(DWF_EINVAL) || !strlen(dwf_status_string(DWF_EINVAL)))
        return fail("status string");
    /* argument checks that come before any device work */
    if (dwf_create(&h, NULL, sub, 8, 1.5, 0.5, 1.8, 0.1, NULL, 0, NULL) != DWF_EINVAL || h)
        return fail("null gauge accepted");
    if (dwf_create(&h, g, odd, 8, 1.5, 0.5, 1.8, 0.1, NULL, 0, NULL) != DWF_EINVAL || h)
        return fail("odd extent accepted");
    if (dwf_create(&h, g, sub, 0, 1.5, 0.5, 1.8, 0.1, NULL, 0, NULL) != DWF_EINVAL || h)
        return fail("Ls = 0 accepted");
    {
        /* a partitioned extent needs lattice - block >= 4 (the snake halo),
           blocks must divide the lattice and be even */
        const int dims[4] = {8, 4, 4, 4};
        const int narrow[4] = {6, 4, 4, 4}, ragged[4] = {3, 4, 4, 4}, odd_blk[4] = {4, 4, 4, 2};
        if (dwf_create(&h, g, dims, 4, 1.5, 0.5, 1.8, 0.1, narrow, 0, NULL) != DWF_EINVAL || h)
            return fail("block that does not divide accepted");
        if (dwf_create(&h, g, dims, 4, 1.5, 0.5, 1.8, 0.1, ragged, 0, NULL) != DWF_EINVAL || h)
            return fail("odd block accepted");
        if (dwf_create(&h, g, dims, 4, 1.5, 0.5, 1.8, 0.1, odd_blk, 0, NULL) != DWF_EINVAL || h)
            return fail("block too large for the snake halo accepted");
    }
    if (dwf_fma_peak(NULL, DWF_F32, &t) != DWF_EINVAL) return fail("null handle accepted");
    if (strcmp(dwf_last_error(NULL), "null handle") != 0) return fail("last error of null");
    if (dwf_kernel_launch_count() != 0) return fail("launches without a device call");
    printf("ok\n");
    return 0;
}
"""


def test_header_is_plain_c_and_a_c_client_links(tmp_path):
    """include/dwf.h compiles as strict C99 (no C++ in the ABI), a C program
    links against the library and its host-side calls behave as documented."""
    import shutil
    import subprocess
    import pytest
    from paper_2104_05615_gb300 import build
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lib_path = build.build()
    src = tmp_path / "client.c"
    src.write_text(C_CLIENT)
    exe = tmp_path / "client"
    lib_dir = os.path.dirname(lib_path)
    cmd = [cc, "-std=c99", "-pedantic", "-Wall", "-Wextra", "-Werror",
           "-I" + os.path.join(ROOT, "include"), str(src), "-o", str(exe),
           "-L" + lib_dir, "-ldwf_gb300", "-Wl,-rpath," + lib_dir]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stderr


def _brute_regions(dims, sub):
    """Per block (the one at the origin): even interior sites, odd sites within
    L1 distance 1 and even sites within L1 distance 2 of it, counted over the
    whole periodic lattice (the block is a box, so the distance is the sum of
    the per-dimension distances to its interval)."""
    import numpy as np
    grids = np.meshgrid(*[np.arange(L) for L in dims], indexing="ij")
    dist = np.zeros(dims, dtype=np.int64)
    for mu, (L, S) in enumerate(zip(dims, sub)):
        y = grids[mu]
        if S == L:
            continue
        inside = y < S
        d = np.minimum((y - (S - 1)) % L, (-y) % L)
        dist += np.where(inside, 0, d)
    par = sum(grids) % 2
    return (int(((dist == 0) & (par == 0)).sum()), int(((dist <= 1) & (par == 1)).sum()),
            int(((dist <= 2) & (par == 0)).sum()))


def test_query_geometry_regions_match_brute_force():
    """dwf_query_geometry (host-only) against a brute-force count of the
    snake-term regions (Sec. 2.3 / 3.1.2): the even interior, the odd sites
    one hop out and the even sites two hops out, for the workloads' block
    shapes; refused shapes give DWF_EINVAL."""
    import numpy as np
    import pytest
    from paper_2104_05615_gb300 import binding as B
    cases = [((16, 16, 16, 32), (8, 8, 8, 8)), ((32, 32, 32, 64), (16, 16, 16, 16)),
             ((8, 8, 8, 8), (4, 4, 4, 4)), ((12, 12, 12, 12), (4, 4, 4, 4)),
             ((8, 8, 8, 16), (4, 4, 4, 4)), ((8, 4, 4, 4), (4, 4, 4, 4)),
             ((12, 2, 2, 2), (6, 2, 2, 2)), ((6, 2, 2, 2), (6, 2, 2, 2))]
    for dims, sub in cases:
        g = B.dwf_query_geometry(dims, sub)
        interior, o1, e2 = _brute_regions(dims, sub)
        nblk = int(np.prod(dims) // np.prod(sub))
        assert g["blocks"] == nblk and g["even_sites"] == np.prod(dims) // 2, (dims, sub)
        assert (g["block_sites"], g["o1_sites"], g["e2_sites"]) == (interior, o1, e2), (dims, sub, g)
        for k in ("block_sites", "o1_sites", "e2_sites"):
            assert g[k + "_padded"] >= g[k] and g[k + "_padded"] % 32 == 0, (dims, sub, k)
    assert B.dwf_query_geometry((6, 2, 2, 2)) == B.dwf_query_geometry((6, 2, 2, 2), (6, 2, 2, 2))
    for dims, sub in (((4, 4, 4, 4), (2, 4, 4, 4)), ((8, 4, 4, 4), (6, 4, 4, 4)),
                      ((3, 4, 4, 4), None), ((8, 4, 4, 4), (4, 4, 4, 3))):
        with pytest.raises(B.DwfError) as e:
            B.dwf_query_geometry(dims, sub)
        assert e.value.status == B.DWF_EINVAL
