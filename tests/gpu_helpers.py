"""Shared helpers of the GPU parity tests: run an instance through the C ABI
and compare with the oracle at the stated tolerances."""
import numpy as np

import oracle

# tolerances of the plain FP64 path against the oracle
REL_ROWS = 1e-10      # moments mu and concentration C, relative, every output time
REL_N = 1e-9          # distribution: L-inf error <= REL_N * max(n)


def gpu_solve(inst, path="plain", device_buffers=True, window=-1):
    import torch
    import paper_2411_00742_gb300 as P
    g = P.Grid.from_problem(inst.problem, path=path)
    g.set_window(window)
    if device_buffers:
        g.set_state(torch.as_tensor(np.ascontiguousarray(inst.n0)).cuda(), inst.C0, inst.t0)
        rows_t = torch.zeros((len(inst.t_out), P.ncols(inst.problem.ndim)), dtype=torch.float64, device="cuda")
        _, steps = g.solve(inst.t_out, out=rows_t)
        rows = rows_t.cpu().numpy()
        n_t = torch.zeros(inst.problem.ncells, dtype=torch.float64, device="cuda")
        _, C, t = g.get_state(out=n_t)
        n = n_t.cpu().numpy()
    else:
        g.set_state(np.ascontiguousarray(inst.n0), inst.C0, inst.t0)
        rows, steps = g.solve(inst.t_out)
        n, C, t = g.get_state()
    g.close()
    return dict(rows=rows, steps=steps, n=n, C=C, t=t)


def assert_rows_close(got, want, rel=REL_ROWS):
    assert got.shape == want.shape
    np.testing.assert_allclose(got[:, 0], want[:, 0], rtol=1e-12, atol=0)
    ref = want[:, 1:]
    err = np.abs(got[:, 1:] - ref)
    bound = rel * np.abs(ref)
    bad = err > bound
    assert not bad.any(), f"max rel err {np.max(err / np.maximum(np.abs(ref), 1e-300)):.3e} at {np.argwhere(bad)[:5]}"


def assert_n_close(got, want, rel=REL_N):
    scale = np.max(np.abs(want))
    err = np.max(np.abs(np.asarray(got).reshape(want.shape) - want))
    assert err <= rel * scale, f"L-inf error {err:.3e} > {rel:.0e} * max(n) = {rel * scale:.3e}"


def compare_instance(inst, path="plain", device_buffers=True, window=-1):
    want = oracle.solve_instance(inst)
    got = gpu_solve(inst, path=path, device_buffers=device_buffers, window=window)
    assert got["steps"] == want["steps"], (got["steps"], want["steps"])
    assert_rows_close(got["rows"], want["rows"])
    assert_n_close(got["n"], want["n"])
    assert abs(got["C"] - want["C"]) <= REL_ROWS * abs(want["C"])
    return got, want
