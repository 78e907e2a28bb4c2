"""Two Philox4x32-10 implementations that are not ours, for pinning the oracle.

* cuRAND's host generator (CURAND_RNG_PSEUDO_PHILOX4_32_10 = 161) runs on the
  CPU.  Its output block b (four words) is Philox of counter
  (b // 65536, 0, b % 65536, 0) under key (seed lo, seed hi): the host
  generator emulates 65536 threads, thread s on subsequence s.  That mapping
  was found by matching blocks, not assumed; the test checks it on every
  block it uses.
* Triton's Philox (``tl.philox``) run by Triton's CPU interpreter, which takes
  all four counter words and a 64-bit seed.  It runs in a subprocess because
  the interpreter is switched on by an environment variable read at import.
"""
import ctypes
import ctypes.util
import json
import os
import subprocess
import sys

import numpy as np

CURAND_RNG_PSEUDO_PHILOX4_32_10 = 161


def _curand():
    for name in ("/usr/local/cuda/lib64/libcurand.so", ctypes.util.find_library("curand")):
        if not name:
            continue
        try:
            return ctypes.CDLL(name)
        except OSError:
            pass
    return None


def curand_host_blocks(seed: int, n_blocks: int):
    """First n_blocks four-word blocks of cuRAND's host Philox generator, or None."""
    lib = _curand()
    if lib is None:
        return None
    g = ctypes.c_void_p()
    if lib.curandCreateGeneratorHost(ctypes.byref(g), CURAND_RNG_PSEUDO_PHILOX4_32_10) != 0:
        return None
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(g, ctypes.c_ulonglong(seed)) == 0
        out = np.zeros(4 * n_blocks, dtype=np.uint32)
        assert lib.curandGenerate(g, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(out.size)) == 0
    finally:
        lib.curandDestroyGenerator(g)
    return out.reshape(n_blocks, 4)


def curand_block_counters(n_blocks: int) -> np.ndarray:
    b = np.arange(n_blocks, dtype=np.uint64)
    ctr = np.zeros((n_blocks, 4), dtype=np.uint32)
    ctr[:, 0] = (b // 65536).astype(np.uint32)
    ctr[:, 2] = (b % 65536).astype(np.uint32)
    return ctr


_TRITON_SCRIPT = r"""
import os, sys, json
os.environ["TRITON_INTERPRET"] = "1"
import numpy as np, torch, triton, triton.language as tl

@triton.jit
def _philox_kernel(out_ptr, seed, c0_ptr, c1_ptr, c2_ptr, c3_ptr, n: tl.constexpr):
    i = tl.arange(0, n)
    a, b, c, d = tl.philox(seed, tl.load(c0_ptr + i), tl.load(c1_ptr + i),
                           tl.load(c2_ptr + i), tl.load(c3_ptr + i), 10)
    tl.store(out_ptr + 4 * i, a)
    tl.store(out_ptr + 4 * i + 1, b)
    tl.store(out_ptr + 4 * i + 2, c)
    tl.store(out_ptr + 4 * i + 3, d)

req = json.loads(sys.stdin.read())
res = []
for item in req:
    seed = int(item["seed"])
    ctr = np.array(item["ctr"], dtype=np.uint32).reshape(-1, 4)
    n = len(ctr)
    cs = [torch.from_numpy(np.ascontiguousarray(ctr[:, w]).view(np.int32)) for w in range(4)]
    out = torch.zeros(4 * n, dtype=torch.int32)
    _philox_kernel[(1,)](out, seed, *cs, n)
    res.append(out.numpy().view(np.uint32).tolist())
print(json.dumps(res))
"""


def triton_philox(requests):
    """requests: list of (seed, ctr[n,4]) with n a power of two.  Returns list of
    (n,4) uint32 arrays, or None if Triton's interpreter is unavailable."""
    try:
        import triton  # noqa: F401
    except Exception:
        return None
    payload = json.dumps([{"seed": int(s), "ctr": np.asarray(c, dtype=np.uint32).reshape(-1).tolist()}
                          for s, c in requests])
    env = dict(os.environ, TRITON_INTERPRET="1")
    p = subprocess.run([sys.executable, "-c", _TRITON_SCRIPT], input=payload, capture_output=True,
                       text=True, env=env, timeout=600)
    if p.returncode != 0:
        raise RuntimeError(p.stderr[-2000:])
    return [np.array(r, dtype=np.uint32).reshape(-1, 4) for r in json.loads(p.stdout)]
