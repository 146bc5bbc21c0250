"""The C ABI is usable from plain C: a C99 program that includes include/coolchic.h
compiles without warnings, takes the address of every declared entry point, links
against the built library and calls the entry points that need no GPU."""
import os
import re
import shutil
import subprocess

import pytest

from paper_2403_11651_gb300 import build as _build
from paper_2403_11651_gb300 import coolchic as cc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "coolchic.h")

PROGRAM = r"""
#include <stdio.h>
#include <string.h>
#include "coolchic.h"

typedef void (*any_fn)(void);
static any_fn table[] = { %(table)s };

int main(void) {
    cc_config cfg;
    int n = 0, e;
    memset(&cfg, 0, sizeof cfg);
    cfg.levels = 7; cfg.arm_ctx = 24; cfg.arm_layers = 2; cfg.up_kernel = 8;
    cfg.up_per_level = 1; cfg.syn_hidden = 40; cfg.syn_res3x3 = 2;
    cfg.lam = 1e-3f; cfg.lr = 1e-2f; cfg.total_iters = 100; cfg.ste_frac = 0.2f;
    if ((e = cc_param_count(&cfg, &n)) != CC_OK) return 10;
    printf("params %%d\n", n);
    if ((e = cc_latent_count(&cfg, 512, 768, &n)) != CC_OK) return 11;
    printf("latents %%d\n", n);
    if (cc_latent_count(&cfg, 0, 768, &n) != CC_EINVAL) return 12;
    cfg.arm_ctx = 7;
    if (cc_param_count(&cfg, &n) != CC_EINVAL) return 13;
    if (cc_warm_param_count(&n) != CC_OK) return 14;
    printf("warm %%d\n", n);
    printf("strerror %%s\n", cc_strerror(CC_ETIMEOUT));
    printf("entry_points %%d\n", (int)(sizeof table / sizeof table[0]));
    return 0;
}
"""


def _declared():
    with open(HEADER) as f:
        text = f.read()
    return sorted(set(re.findall(r"^\s*(?:int|void|const char\*)\s+(cc_\w+)\s*\(", text, re.M)))


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_plain_c_program_links_and_runs(tmp_path):
    cc.load()
    names = _declared()
    src = tmp_path / "abi.c"
    src.write_text(PROGRAM % {"table": ", ".join(f"(any_fn){n}" for n in names)})
    exe = tmp_path / "abi"
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror",
                    f"-I{os.path.dirname(HEADER)}", str(src), "-o", str(exe),
                    f"-L{_build.BUILD}", "-lcoolchic", f"-Wl,-rpath,{_build.BUILD}"],
                   check=True, capture_output=True, text=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    lines = dict(line.split(" ", 1) for line in out.strip().splitlines())
    assert int(lines["params"]) == cc.cc_param_count(cc.make_config(cc.load_config("c2")))
    assert int(lines["latents"]) == 524256
    assert int(lines["warm"]) == 28800
    assert lines["strerror"] == cc.cc_strerror(cc.CC_ETIMEOUT)
    assert int(lines["entry_points"]) == len(names) >= 30
