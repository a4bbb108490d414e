"""Failure detection without a GPU fault (marked gpu).

The device checks every rounded value's distance to its integer against the plan's
a-priori bound and raises a status flag that the host turns into TM_EPRECISION. A
correct bound never trips it, so the test injects the failure on the host: a child
process runs with TRUNCMUL_FAULT_EMAX_SCALE set, which scales every bound the device
sees down by 10^-12. Every entry point must then report TM_EPRECISION (synchronous
calls, the asynchronous status query, host buffers, kept operands, batches, the
request loop, division, the allocation-free entry point) while the products
themselves stay the exact ones a normal process computes; in a normal process the
same calls succeed. The allocation-free entry point reads its status word through
its own branch (copy, clear, wait); a later call on a zero operand must report
TM_OK, which shows that branch left the word cleared."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

import workloads
from gpu_util import dev, host

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
N_BITS = 100003
N_STATIC = 60001          # tm_mul_static's sizes stop at 65536 bits

CHILD = r'''
import json, sys
sys.path.insert(0, sys.argv[1]); sys.path.insert(0, sys.argv[1] + "/tests")
import numpy as np, torch
import paper_1703_00640_gb300 as pkg
import workloads
pkg.load()
n = int(sys.argv[2])
u, v = workloads.pattern_limbs("random", n, seed=3)
du = torch.from_numpy(u.view(np.int64)).cuda()
dv = torch.from_numpy(v.view(np.int64)).cuda()
res = {"codes": {}, "out": {}}
def code(fn):
    try:
        fn()
        return 0
    except pkg.TruncMulError as e:
        return e.code
for kind in ("lo", "hi", "full"):
    out, rep = pkg.mul(kind, du, dv, n, check=False)
    res["codes"]["sync_" + kind] = rep["status"]
    res["out"][kind] = out.cpu().numpy().view(np.uint64).tolist()
s = torch.cuda.Stream()
pkg.mul("lo", du, dv, n, stream=s, report=False)
res["codes"]["async_status"] = pkg.stream_status(s)["rc"]
res["codes"]["host"] = code(lambda: pkg.mul_host("hi", u, v, n))
op = pkg.Operand("lo", dv, n)
res["codes"]["operand"] = code(lambda: op.mul(du))
op.close()
items = [("lo", n, torch.empty(pkg.out_limbs("lo", n), dtype=torch.int64, device="cuda"), du, dv),
         ("hi", 3000, torch.empty(pkg.out_limbs("hi", 3000), dtype=torch.int64, device="cuda"),
          du[: (3000 + 63) // 64], dv[: (3000 + 63) // 64])]
b = pkg.Batch(items)
b.launch()
res["codes"]["batch"] = b.status()["rc"]
b.close()
srv = pkg.Server(budget_bytes=1 << 30, slots=2)
outs = [torch.empty(pkg.out_limbs("hi", n), dtype=torch.int64, device="cuda") for _ in range(2)]
for o in outs:
    srv.submit("hi", o, du, dv, n)
done = []
while len(done) < 2:
    done += srv.progress()
srv.close()
res["codes"]["server"] = sorted(st for _, st in done)
m = u.copy()
k = 64 * (m.size - 1)
m = m[: k // 64]
m[-1] |= np.uint64(1 << 63)
bar = pkg.Barrett(torch.from_numpy(m.view(np.int64)).cuda(), k)
x = torch.from_numpy(np.concatenate([u[: k // 64], v[: k // 64]]).view(np.int64)).cuda()
res["codes"]["divrem"] = code(lambda: bar.divrem(x))
bar.close()
ns = int(sys.argv[3])
us, vs = workloads.pattern_limbs("random", ns, seed=4)
dus = torch.from_numpy(us.view(np.int64)).cuda()
dvs = torch.from_numpy(vs.view(np.int64)).cuda()
for kind in ("lo", "hi", "full"):
    o = torch.full((pkg.out_limbs(kind, ns),), -1, dtype=torch.int64, device="cuda")
    rc, _ = pkg.mul_static(kind, dus, dvs, ns, o)
    res["codes"]["static_" + kind] = rc
    res["out"]["static_" + kind] = o.cpu().numpy().view(np.uint64).tolist()
# a zero operand rounds every coefficient exactly (distance 0), so this call
# reports TM_OK only if the flagged calls before it left the status word cleared
o = torch.empty(pkg.out_limbs("lo", ns), dtype=torch.int64, device="cuda")
rc, _ = pkg.mul_static("lo", torch.zeros_like(dus), dvs, ns, o)
res["codes"]["static_clear_after"] = rc
print(json.dumps(res))
'''


def _child(scale):
    env = dict(os.environ)
    env.pop("TRUNCMUL_FAULT_EMAX_SCALE", None)
    if scale is not None:
        env["TRUNCMUL_FAULT_EMAX_SCALE"] = scale
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT, str(N_BITS), str(N_STATIC)], env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


@pytest.fixture(scope="module")
def pkg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1703_00640_gb300 as p
    p.build()
    p.load()
    return p


def test_injected_margin_failure_is_reported_everywhere(pkg):
    res = _child("1e-12")
    E = pkg.TM_EPRECISION
    codes = res["codes"]
    for key in ("sync_lo", "sync_hi", "sync_full", "async_status", "host", "operand",
                "batch", "divrem", "static_lo", "static_hi", "static_full"):
        assert codes[key] == E, (key, codes)
    assert codes["server"] == [E, E]
    assert codes["static_clear_after"] == 0, codes
    # the arithmetic is untouched: the limbs equal this (uninjected) process's
    u, v = workloads.pattern_limbs("random", N_BITS, seed=3)
    for kind in ("lo", "hi", "full"):
        ref, rep = pkg.mul(kind, dev(u), dev(v), N_BITS)
        assert rep["status"] == 0
        assert np.array_equal(np.array(res["out"][kind], dtype=np.uint64), host(ref)), kind
    import torch
    us, vs = workloads.pattern_limbs("random", N_STATIC, seed=4)
    for kind in ("lo", "hi", "full"):
        o = torch.empty(pkg.out_limbs(kind, N_STATIC), dtype=torch.int64, device="cuda")
        rc, _ = pkg.mul_static(kind, dev(us), dev(vs), N_STATIC, o)
        assert rc == 0
        got = np.array(res["out"]["static_" + kind], dtype=np.uint64)
        assert np.array_equal(got, host(o)), "static " + kind


@pytest.mark.parametrize("scale", [None, "2", "0", "junk"])
def test_without_injection_every_call_succeeds(pkg, scale):
    """No variable, or a value outside (0, 1] (ignored): every status is TM_OK."""
    codes = _child(scale)["codes"]
    for key, c in codes.items():
        assert c == ([0, 0] if key == "server" else 0), (key, codes)


BARRIER_CHILD = r'''
import json, sys
sys.path.insert(0, sys.argv[1]); sys.path.insert(0, sys.argv[1] + "/tests")
import numpy as np, torch
import paper_1703_00640_gb300 as pkg
import workloads
pkg.load()
n = 65536
u, v = workloads.pattern_limbs("random", n, seed=8)
du = torch.from_numpy(u.view(np.int64)).cuda()
dv = torch.from_numpy(v.view(np.int64)).cuda()
res = {}
pkg.set_fused(pkg.FUSED_ALWAYS)
_, rep = pkg.mul("lo", du, dv, n, check=False)
res["single"] = rep["status"]
items = [("hi", 40000 + 97 * i, torch.empty(pkg.out_limbs("hi", 40000 + 97 * i),
          dtype=torch.int64, device="cuda"), du[:(40000 + 97 * i + 63) // 64],
          dv[:(40000 + 97 * i + 63) // 64]) for i in range(8)]
b = pkg.Batch(items)                     # created in mode 2: one persistent launch
b.launch()
res["batch"] = b.status()["rc"]
b.close()
pkg.set_fused(pkg.FUSED_NEVER)           # per-phase launches: no barrier, no injection
out, rep = pkg.mul("lo", du, dv, n, check=False)
res["after"] = rep["status"]
res["after_out"] = out.cpu().numpy().view(np.uint64).tolist()
print(json.dumps(res))
'''


def test_barrier_timeout_is_reported_and_the_device_stays_usable(pkg):
    """TRUNCMUL_FAULT_BARRIER=1: the last CTA of a single-launch product leaves at
    the first grid barrier, and the first unit of a persistent batch is never
    reported as finished; the others' bounded waits run out (about a second) and the
    calls report TM_ETIMEOUT. A per-phase product
    in the same process afterwards succeeds with the exact limbs."""
    env = dict(os.environ)
    env["TRUNCMUL_FAULT_BARRIER"] = "1"
    env.pop("TRUNCMUL_FAULT_EMAX_SCALE", None)
    r = subprocess.run([sys.executable, "-c", BARRIER_CHILD, ROOT], env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    res = json.loads(r.stdout.strip().splitlines()[-1])
    assert res["single"] == pkg.TM_ETIMEOUT, res
    assert res["batch"] == pkg.TM_ETIMEOUT, res
    assert res["after"] == 0
    u, v = workloads.pattern_limbs("random", 65536, seed=8)
    ref, _ = pkg.mul("lo", dev(u), dev(v), 65536)
    assert np.array_equal(np.array(res["after_out"], dtype=np.uint64), host(ref))
