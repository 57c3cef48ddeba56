"""Statistical validation as in the paper (Sec. III): the mean of the
estimator over many realisations of the quadratic non-Gaussian
redshift-space field must agree with [B_l^m]_d, the model bispectrum of
Eqs. mod_bs/rsd_bs at each combination's mean wavevectors, binned as the
estimator (the oracle's discrete model), within the scatter of the
realisations.

Setup of the paper's run: N_g = 384, L = 215, P = A k^-2 with sigma_G =
0.1, f_NG = 0.5, beta = 1, 50 realisations, k1 = 2.1 +- 0.1, here with
(mu, t) bins of 0.05 and all 16 moments l <= 6.  Per moment, with z the
pull (mean - model) / (sigma / sqrt(50)) over the populated bins: chi^2
per bin below 2, mean pull within 0.6 (five times its own standard error
for 70 bins), at least 90% of the bins within 3 sigma.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2405_14513_gb300 import synth

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2405_14513_gb300 import api  # noqa: E402


def test_mean_over_realisations_matches_discrete_model():
    ng, L, edges, nmu, lmax = 384, 215.0, np.array([2.0, 2.2]), 10, 6
    sigma_g, f_ng, beta, seeds, batch = 0.1, 0.5, 1.0, 50, 10
    plan = api.Plan(ng, L, edges, nmu, nmu, lmax, precision="mixed_tc", max_batch=batch)
    ws = plan.workspace(batch)
    out = []
    for s0 in range(0, seeds, batch):
        f = torch.stack([synth.make_field_torch(ng, L, 1 + s, sigma_g=sigma_g, f_ng=f_ng, beta=beta,
                                                device="cuda").float() for s in range(s0, s0 + batch)])
        out.append(plan.estimate(f.contiguous(), ws).cpu().numpy())
        assert plan.workspace_status(ws, batch) == 0
    plan.close()
    B = np.concatenate(out)[:, 0]                                   # [seed][mu][t][lm]
    A = synth.power_amplitude(ng, L, sigma_g, -2.0)
    model = O.select_even(O.discrete_model(ng, L, edges, nmu, nmu, lmax, A, -2.0, f_ng, beta), lmax)[0]
    mean, sem = B.mean(0), B.std(0, ddof=1) / np.sqrt(seeds)
    lines = []
    for i, (l, m) in enumerate(O.even_moments(lmax)):
        fin = np.isfinite(model[..., i]) & np.isfinite(mean[..., i])
        assert fin.sum() >= 50, (l, m)
        z = (mean[..., i] - model[..., i])[fin] / sem[..., i][fin]
        chi2, mz, f3 = np.mean(z ** 2), z.mean(), np.mean(np.abs(z) < 3)
        lines.append(f"B_{l}^{m}: bins {fin.sum()}, chi2/bin {chi2:.2f}, mean pull {mz:+.2f}, within 3 sigma {f3:.2f}")
        assert chi2 < 2.0 and abs(mz) < 0.6 and f3 >= 0.9, lines[-1]
    print("\n".join(lines))
