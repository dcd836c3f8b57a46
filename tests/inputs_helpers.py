"""Small helpers shared by GPU tests: wrap device-generated arrays as an inputs.Problem (host
copies), so that the oracle can smooth exactly the bytes the CUDA path consumed."""
import numpy as np

from paper_2502_11686_gb300 import inputs


def as_problem(k, n, m, F, H, K, G, C, o):
    h = lambda t: np.ascontiguousarray(t.cpu().numpy())   # noqa: E731
    return inputs.Problem(k=k, n=n, m=np.full(k, m, np.int32), F=h(F), H=h(H), c=None, K=h(K),
                          G=h(G).reshape(-1), o=h(o).reshape(-1), C=h(C).reshape(-1),
                          name=f"device-generated k={k} n={n} m={m}")
