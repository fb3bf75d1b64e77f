"""How strong the oracle pins are: plant one plausible mistake at a time in an oracle source (a
dropped term, a wrong sign, a swapped operand, an off-by-one bound, a changed table constant),
run that oracle's `-m "not gpu"` pins, and restore the source.  Every mistake must make at least
one pin fail ("CAUGHT"); a "MISSED" line names a pin that is missing.  CPU only; the oracle
sources are edited in place, so the script refuses to start over uncommitted changes to them.

Usage: python tests/mutate_oracles.py [name ...]     (no names: every mutation; a few minutes)
"""
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
C = "oracle/potr_oracle.c"

MUT = [
    # removal effect
    ("pd_mul", C, "(PK - P[3 * (i + 1) + ch]) / (1.0 - a)) - PK;\n          dse +=",
     "(PK - P[3 * (i + 1) + ch]) * (1.0 - a)) - PK;\n          dse +="),
    ("dse_factor", C, "dse += pd * pd + 2.0 * pd * diff[ch];", "dse += pd * pd + pd * diff[ch];"),
    ("dse_sign", C, "dse += pd * pd + 2.0 * pd * diff[ch];", "dse += pd * pd - 2.0 * pd * diff[ch];"),
    ("imp_alpha", C, "double w = Tv[i] * a;", "double w = a;"),
    ("imp_tnext", C, "        Tv[i] = T;\n", "        Tv[i] = T * (1.0 - a);\n"),
    # compositing walk
    ("tmin_after", C, "    if (Tn < cfg->t_min) break;\n",
     "    if (Tn < cfg->t_min) { out[K].pos = i - s; out[K].k = k; out[K].alpha = a; ++K; last = i - s + 1; T = Tn; break; }\n"),
    ("tmin_continue", C, "    if (Tn < cfg->t_min) break;\n", "    if (Tn < cfg->t_min) continue;\n"),
    ("amin_le", C, "    if (a < cfg->alpha_min) continue;\n", "    if (a < 0.5f * cfg->alpha_min) continue;\n"),
    ("amax_drop", C, "float a = fminf(cfg->alpha_max, sp->opacity[k] * G);", "float a = fminf(1.0f, sp->opacity[k] * G);"),
    ("cross_sign", C, "float u = fmaf(A, dx, B * dy);", "float u = fmaf(A, dx, -B * dy);"),
    ("comp_T", C, "    for (int ch = 0; ch < 3; ++ch) c[ch] += T * a * sp->rgb[ch * sp->n + ent[i].k];\n    T *= (1.0 - a);",
     "    for (int ch = 0; ch < 3; ++ch) c[ch] += T * a * sp->rgb[ch * sp->n + ent[i].k];\n    T *= (1.0 - 0.5 * a);"),
    ("comp_noT", C, "c[ch] += T * a * sp->rgb[ch * sp->n + ent[i].k];", "c[ch] += a * sp->rgb[ch * sp->n + ent[i].k];"),
    ("centre_half", C, "int64_t K = walk_pixel(&job->sp, cfg, job->vals, s, e, (float)x + 0.5f, (float)y + 0.5f, -1, ent,",
     "int64_t K = walk_pixel(&job->sp, cfg, job->vals, s, e, (float)x, (float)y + 0.5f, -1, ent,"),
    # activation
    ("rot_sign", C, "R[0][1] = 2.0f * (qx * qy - qw * qz);", "R[0][1] = 2.0f * (qx * qy + qw * qz);"),
    ("rot_transpose", C, "M[i][j] = R[i][j] * s[j];", "M[i][j] = R[j][i] * s[j];"),
    ("scale_row", C, "M[i][j] = R[i][j] * s[j];", "M[i][j] = R[i][j] * s[i];"),
    ("scale_ln", C, "s[a] = orc_exp2r(log_scales[a * n + k] * kLog2e);", "s[a] = orc_exp2r(log_scales[a * n + k]);"),
    ("sigmoid_flip", C, "opacity[k] = 1.0f / (1.0f + ex);", "opacity[k] = ex / (1.0f + ex);"),
    ("qnorm_drop", C, "qw = qw / r; qx = qx / r; qy = qy / r; qz = qz / r;", "(void)r;"),
    # SH
    ("sh_cs_phase", C, "pmm *= -fact * s;", "pmm *= fact * s;"),
    ("sh_sin_cos", C, "else v = sqrt(2.0) * K * sin(am * phi) * P;", "else v = sqrt(2.0) * K * cos(am * phi) * P;"),
    ("sh_sqrt2", C, "else if (m > 0) v = sqrt(2.0) * K * cos(am * phi) * P;", "else if (m > 0) v = K * cos(am * phi) * P;"),
    ("sh_offset", C, "      v += 0.5;\n", "      v += 0.0;\n"),
    ("sh_clamp", C, "rgb[ch * n + k] = v > 0.0 ? v : 0.0;", "rgb[ch * n + k] = v;"),
    ("sh_dir", C, "double d[3] = {(double)mu[0] - cc[0], (double)mu[1] - cc[1], (double)mu[2] - cc[2]};",
     "double d[3] = {cc[0] - (double)mu[0], cc[1] - (double)mu[1], cc[2] - (double)mu[2]};"),
    ("sh_channel", C, "v += (double)sh[(i * 3 + ch) * n + k] * Y[i];", "v += (double)sh[(ch * 16 + i) * n + k] * Y[i];"),
    ("cam_centre", C, "cc[j] = -((double)W[0 * 4 + j] * W[3] + (double)W[1 * 4 + j] * W[7] + (double)W[2 * 4 + j] * W[11]);",
     "cc[j] = -((double)W[j * 4 + 0] * W[3] + (double)W[j * 4 + 1] * W[7] + (double)W[j * 4 + 2] * W[11]);"),
    # projection
    ("lowpass_c", C, "float c = ((U1[0] * T1[0] + U1[1] * T1[1]) + U1[2] * T1[2]) + cfg->lowpass;",
     "float c = ((U1[0] * T1[0] + U1[1] * T1[1]) + U1[2] * T1[2]);"),
    ("jac_sign", C, "float j02 = -(cam->fx * xc) / z2;", "float j02 = (cam->fx * xc) / z2;"),
    ("jac_clamp", C, "float xc = fminf(lim_x, fmaxf(-lim_x, txz)) * t[2];", "float xc = txz * t[2];"),
    ("det_sign", C, "float det = a * c - b * b;", "float det = a * c + b * b;"),
    ("conic_b", C, "float ca = c / det, cb = -b / det, cc2 = a / det;", "float ca = c / det, cb = b / det, cc2 = a / det;"),
    ("conic_swap", C, "float ca = c / det, cb = -b / det, cc2 = a / det;", "float ca = a / det, cb = -b / det, cc2 = c / det;"),
    ("radius_2s", C, "float r = ceilf(3.0f * sqrtf(lam));", "float r = ceilf(2.0f * sqrtf(lam));"),
    ("qcoef_b", C, "qcoef[n + k] = cb * (-kLog2e);", "qcoef[n + k] = cb * kA;"),
    ("mean_cx", C, "float mx = cam->fx * txz + cam->cx;", "float mx = cam->fx * txz - cam->cx;"),
    ("near_cull", C, "if (!(t[2] > cfg->near_z)) continue;", "if (!(t[2] > 0.0f)) continue;"),
    ("rect_x1", C, "float fx1 = floorf((mx + r) / (float)cfg->tile_w) + 1.0f;", "float fx1 = floorf((mx + r) / (float)cfg->tile_w);"),
    ("view_row", C, "for (int i = 0; i < 3; ++i) t[i] = ((W[i * 4 + 0] * mu[0] + W[i * 4 + 1] * mu[1]) + W[i * 4 + 2] * mu[2]) + W[i * 4 + 3];",
     "for (int i = 0; i < 3; ++i) t[i] = ((W[0 * 4 + i] * mu[0] + W[1 * 4 + i] * mu[1]) + W[2 * 4 + i] * mu[2]) + W[i * 4 + 3];"),
    # binning and sort
    ("sort_unstable", C, "if (ks[b] < ks[a]) {", "if (ks[b] <= ks[a]) {"),
    ("key_order", C, "keys[e] = (tile << 32) | (uint64_t)dbits;", "keys[e] = ((uint64_t)dbits << 32) | tile;"),
    ("rect_colmajor", C, "    for (int32_t ty = rect[n + k]; ty < rect[3 * n + k]; ++ty)\n      for (int32_t tx = rect[k]; tx < rect[2 * n + k]; ++tx) {",
     "    for (int32_t tx = rect[k]; tx < rect[2 * n + k]; ++tx)\n      for (int32_t ty = rect[n + k]; ty < rect[3 * n + k]; ++ty) {"),
    ("cull_margin", C, "float margin = 1e-5f * mag + 1e-4f;", "float margin = -0.05f * mag;"),
    ("cull_centre", C, "if (ux0 <= 0.0f && ux1 >= 0.0f && vy0 <= 0.0f && vy1 >= 0.0f) pmax = fmaxf(pmax, 0.0f);", ""),
    ("cull_edge", C, "float u1 = fminf(fmaxf(ku * vy1, ux0), ux1);", "float u1 = fminf(fmaxf(ku * vy0, ux0), ux1);"),
    ("ranges_first", C, "if (i == 0 || (keys[i - 1] >> 32) != (keys[i] >> 32)) ranges[2 * t] = (uint32_t)i;",
     "if (i == 0 || (keys[i - 1] >> 32) != (keys[i] >> 32)) ranges[2 * t] = (uint32_t)(i + (i > 0));"),
    # second batch
    ("qnorm_term", C, "float n2 = ((qw * qw + qx * qx) + qy * qy) + qz * qz;", "float n2 = (qw * qw + qx * qx) + qy * qy;"),
    ("rot_diag", C, "R[2][2] = 1.0f - 2.0f * (qx * qx + qy * qy);", "R[2][2] = 1.0f - 2.0f * (qx * qx + qz * qz);"),
    ("cov_index", C, "jj[6] = {0, 1, 2, 1, 2, 2};", "jj[6] = {0, 1, 2, 1, 2, 1};"),
    ("sh_norm", C, "factorial(l - am) / factorial(l + am)", "factorial(l + am) / factorial(l - am)"),
    ("legendre_rec", C, "(ll + m - 1.0) * pmm", "(ll + m) * pmm"),
    ("sh_phi", C, "double phi = atan2(y, x);", "double phi = atan2(x, y);"),
    ("proj_row", C, "T0[j] = j00 * W[0 * 4 + j] + j02 * W[2 * 4 + j];", "T0[j] = j00 * W[1 * 4 + j] + j02 * W[2 * 4 + j];"),
    ("eig_disc", C, "float disc = fmaxf(0.1f, mid * mid - det);", "float disc = fmaxf(0.1f, mid * mid + det);"),
    ("eig_minus", C, "float lam = mid + sqrtf(disc);", "float lam = mid - sqrtf(disc);"),
    ("my_fx", C, "float my = cam->fy * tyz + cam->cy;", "float my = cam->fx * tyz + cam->cy;"),
    ("jy_fx", C, "float j11 = cam->fy / t[2];", "float j11 = cam->fx / t[2];"),
    ("rect_y_tw", C, "float fy0 = floorf((my - r) / (float)cfg->tile_h);", "float fy0 = floorf((my - r) / (float)cfg->tile_w);"),
    ("resid_sign", C, "diff[ch] = P[3 * K + ch] - (double)job->target[(int64_t)ch * H * W + pix];",
     "diff[ch] = (double)job->target[(int64_t)ch * H * W + pix] - P[3 * K + ch];"),
    ("tile_transpose", C, "uint64_t tile = tile_base + (uint64_t)ty * (uint64_t)tiles_x + (uint64_t)tx;",
     "uint64_t tile = tile_base + (uint64_t)tx * (uint64_t)tiles_x + (uint64_t)ty;"),
    ("ranges_last", C, "ranges[2 * t + 1] = (uint32_t)(i + 1);", "ranges[2 * t + 1] = (uint32_t)i;"),
    ("tile_ku", C, "float ku = -B / (2.0f * A), kv = -B / (2.0f * C);", "float ku = -B / A, kv = -B / (2.0f * C);"),
    ("brute_sign", C, "acc += d1 * d1 - d0 * d0;", "acc += d0 * d0 - d1 * d1;"),
    ("exp2r_hiclamp", C, "if (y > 125.0f) y = 125.0f;", "if (y > 100.0f) y = 100.0f;"),
    # sixth batch
    ("p_dy_dx", C, "float p = fmaf(u, dx, v * dy);", "float p = fmaf(u, dx, v * dx);"),
    ("v_C_dx", C, "float v = C * dy;", "float v = C * dx;"),
    ("ranges_nobase", C, "int64_t t = (int64_t)((keys[i] >> 32) - tile_base);", "int64_t t = (int64_t)(keys[i] >> 32);"),
    ("vals_nobase", C, "vals[e] = val_base + (uint32_t)k;", "vals[e] = (uint32_t)k;"),
    ("t64_single", C, "if (job->t_final64) job->t_final64[pix] = T64;", "if (job->t_final64) job->t_final64[pix] = (double)T32;"),
    # exp2r
    ("exp2r_coef", C, "  for (int k = 1; k <= 6; ++k) {\n    c = c * ln2;", "  for (int k = 1; k <= 5; ++k) {\n    c = c * ln2;"),
    ("exp2r_round", C, "float n = rintf(y);", "float n = floorf(y);"),
]

TESTS = ["tests/test_oracle_pins.py", "tests/test_oracle_grad.py"]
PR, SH, CO, AD, GR, OI = ("oracle/prune.py", "oracle/sh_compact.py", "oracle/codec.py", "oracle/adam.py",
                          "oracle/grad.py", "oracle/__init__.py")
PY_TESTS = {PR: ["tests/test_oracle_prune.py", "tests/test_oracle_hyperparameters.py"], SH: ["tests/test_oracle_sh_compact.py", "tests/test_oracle_hyperparameters.py"],
            CO: ["tests/test_oracle_codec.py", "tests/test_host_logic.py", "tests/test_oracle_hyperparameters.py"], AD: ["tests/test_oracle_adam.py"], GR: ["tests/test_oracle_grad.py"],
            OI: ["tests/test_oracle_pins.py"]}
MUT += [
    ("m_negsign", PR, "return (math.sqrt(1.0 - (2.0 * a) * x) - 1.0) / a", "return (1.0 - math.sqrt(1.0 - (2.0 * a) * x)) / a"),
    ("m_a", PR, "return (math.sqrt(1.0 - (2.0 * a) * x) - 1.0) / a", "return (math.sqrt(1.0 - a * x) - 1.0) / a"),
    ("cand_le", PR, "dmse[k] < dmse_max_value]", "dmse[k] <= dmse_max_value]"),
    ("budget_r", PR, "// int(remaining)", "// int(remaining + 1)"),
    ("tie_desc", PR, "key=lambda k: (m_map(dmse[k] / dmse_max_value, a), k))", "key=lambda k: (m_map(dmse[k] / dmse_max_value, a), -k))"),
    ("budget_lt", PR, "if budget <= total:", "if budget < total:"),
    ("dmax_q", PR, "10.0 ** (-8.8 - 2.0 * q)", "10.0 ** (-8.8 - q)"),
    ("alive_ign", PR, "if alive[k] and dmse[k] < dmse_max_value]", "if dmse[k] < dmse_max_value]"),
    ("qnan", PR, "imp = np.where(imp >= 0.0, imp, 0.0)", "imp = np.where(np.isnan(imp), 0.0, imp)"),
    ("lam_dc", SH, "np.where(A == 0, 0.0, lam)", "lam"),
    ("lam_chroma", SH, "lams = (lam, 3.0 * lam, 3.0 * lam)", "lams = (lam, lam, lam)"),
    ("cos_abs", SH, "if any(abs(G[i, j]) / math.sqrt(G[i, i] * G[j, j]) > alpha for j in kept):",
     "if any(G[i, j] / math.sqrt(G[i, i] * G[j, j]) > alpha for j in kept):"),
    ("cos_all", SH, "> alpha for j in kept):", "> alpha for j in range(i)):"),
    ("w_sum", SH, "w = np.where(w > 0, w, 0.0) / np.max(w)", "w = np.where(w > 0, w, 0.0) / np.sum(w)"),
    ("w_rows", SH, "rows.append(ws * Y)", "rows.append(Y)"),
    ("pass2_luma", SH, "if not quantises_to_zero(first[i, ch], sf)]", "if not quantises_to_zero(first[i, 0], sf)]"),
    ("quant_floor", SH, "return math.floor(0.5 + x * sf) == 0", "return math.floor(x * sf) == 0"),
    ("dir_rev", SH, "d = np.asarray(mean, np.float64) - c", "d = c - np.asarray(mean, np.float64)"),
    ("alpha_q", SH, "\"alpha\": 1.0 / (1.0 + math.exp(-3.0 * q))", "\"alpha\": 1.0 / (1.0 + math.exp(-q))"),
    ("offset_in", SH, "cols.append(ws * (Y @ L_rgb))", "cols.append(ws * (Y @ L_rgb + 0.5))"),
    ("co_sign", SH, "[0.5, 0.0, -0.5], [-0.25", "[0.5, 0.0, 0.5], [-0.25"),
    ("pass2_skip", SH, "second[:, ch] = _ridge(G, b[:, ch], keep2, lams[ch])", "second[:, ch] = first[:, ch]"),
    ("q_round", CO, "return np.floor(0.5 + np.asarray(x, np.float64) * sf).astype(np.int64)",
     "return np.floor(np.asarray(x, np.float64) * sf).astype(np.int64)"),
    ("root_min", CO, "S = float((mu.max(axis=1) - lo).max())", "S = float((mu.max(axis=1) - lo).min())"),
    ("tol_min", CO, "return np.maximum(gamma, beta * np.min(np.array(d), axis=0))", "return np.maximum(gamma, beta * np.max(np.array(d), axis=0))"),
    ("leaf_centre_corner", CO, "return np.array([corner[a] + (cell[a] + 0.5) * w for a in range(3)])", "return np.array([corner[a] + cell[a] * w for a in range(3)])"),
    ("split_le", CO, "must_split = not (dist < tol[k])", "must_split = not (dist < 2.0 * tol[k])"),
    ("morton", CO, "cx, cy, cz = ((int(X[a, k]) >> sh) & 1 for a in range(3))", "cz, cy, cx = ((int(X[a, k]) >> sh) & 1 for a in range(3))"),
    ("leaf_order", CO, "for k in sorted(members):", "for k in sorted(members, reverse=True):"),
    ("quat_flip", CO, "qn = np.where(qn[0] < 0.0, -qn, qn)", "qn = qn"),
    ("dc_diff", CO, "out[\"sh\"][:3] = np.diff(", "out[\"sh\"][3:6] = np.diff("),
    ("sf_op", CO, "\"sf_opacity\": 1.0 + 200.0 * q", "\"sf_opacity\": 1.0 + 100.0 * q"),
    ("op_offset", CO, "opacity = (op[0] + 0.25) / sf_op", "opacity = (op[0] + 0.5) / sf_op"),
    ("dup_count", CO, "dups.append((leaves[0], len(members) - 1))", "dups.append((leaves[0], len(members)))"),
    ("w_recon", CO, "w = np.sqrt(np.maximum(0.0, 1.0 - (xyz ** 2).sum(axis=0)))", "w = np.sqrt(np.maximum(0.0, 1.0 - xyz.sum(axis=0)))"),
    ("adam_bc1", AD, "p -= (lr / bc1) * m / denom", "p -= lr * m / denom"),
    ("adam_eps", AD, "denom = np.sqrt(v) / np.sqrt(bc2) + eps", "denom = np.sqrt(v / bc2 + eps)"),
    ("qbits", PR, "Q_BITS = 40", "Q_BITS = 30"),
    ("cell_clip", CO, "return np.clip(X, 0, (1 << DEPTH) - 1).astype(np.int64)", "return np.clip(X, 0, (1 << DEPTH)).astype(np.int64)"),
    # third batch
    ("inst_index", C, "job->part_dse[s + ent[i].pos] += dse;", "job->part_dse[s + (uint32_t)i] += dse;"),
    ("nlast_off", C, "    last = i - s + 1;\n", "    last = i - s;\n"),
    ("pass2_dc", SH, "keep2 = [0] + [i for i in kept[1:] if not quantises_to_zero(first[i, ch], sf)]",
     "keep2 = [i for i in kept if not quantises_to_zero(first[i, ch], sf)] or [0]"),
    ("unseen_zero", SH, "return L_rgb @ RGB_TO_YCOCG.T, None, None, None, None", "return np.zeros((16, 3)), None, None, None, None"),
    ("sh_chmajor", CO, "sh = np.asarray(scene.sh, np.float64).reshape(48, -1)[:, order]",
     "sh = np.asarray(scene.sh, np.float64).transpose(1, 0, 2).reshape(48, -1)[:, order]"),
    ("rot_store_w", CO, "\"rotation\": quantise(qn[1:], p[\"sf_rotation\"])", "\"rotation\": quantise(qn[:3], p[\"sf_rotation\"])"),
    ("op_logit", CO, "op = 1.0 / (1.0 + np.exp(-np.asarray(scene.opacity_logits, np.float64)[order]))",
     "op = np.asarray(scene.opacity_logits, np.float64)[order]"),
    ("header_sf", CO, "head += struct.pack(\"<4d\", p[\"sf_scale\"], p[\"sf_rotation\"], p[\"sf_opacity\"], p[\"sf_sh\"])",
     "head += struct.pack(\"<4d\", p[\"sf_rotation\"], p[\"sf_scale\"], p[\"sf_opacity\"], p[\"sf_sh\"])"),
    # fourth batch
    ("kA_scale", C, "const float kA = -0.5f * kLog2e;", "const float kA = -kLog2e;"),
    ("cull_nomargin", C, "float margin = 1e-5f * mag + 1e-4f;", "float margin = 0.0f;"),
    ("cull_max32", C, "#define ORC_CULL_MAX_TILES 64", "#define ORC_CULL_MAX_TILES 32"),
    ("exclude_break", C, "    if ((int64_t)k == exclude) continue;\n", "    if ((int64_t)k == exclude) break;\n"),
    ("near_ge", C, "if (!(t[2] > cfg->near_z)) continue;", "if (!(t[2] >= cfg->near_z)) continue;"),
    # fifth batch
    ("run_remaining", PR, "select(d, i, alive, dmse_max_value, iterations - it, a)", "select(d, i, alive, dmse_max_value, iterations, a)"),
    ("cos_one_minus", SH, "kept = cosine_kept(G, alpha)", "kept = cosine_kept(G, 1.0 - alpha)"),
    ("pass2_lam_luma", SH, "second[:, ch] = _ridge(G, b[:, ch], keep2, lams[ch])", "second[:, ch] = _ridge(G, b[:, ch], keep2, lams[0])"),
    ("dup_range", CO, "for _ in range(1 + extra.get(leaf[0], 0)):", "for _ in range(max(1, extra.get(leaf[0], 0))):"),
    ("tol_sq", CO, "return np.maximum(gamma, beta * np.min(np.array(d), axis=0))", "return np.maximum(gamma, beta * np.min(np.array(d), axis=0) ** 2)"),
    ("g_power_half", GR, "power = -0.5 * (pr[\"ca\"]", "power = -1.0 * (pr[\"ca\"]"),
    ("adam_bc2", AD, "bc2 = 1.0 - b2 ** t", "bc2 = 1.0 - b2 ** (t + 1)"),
    ("dmse_3P", OI, "out += d / (3.0 * cam.pixels) / n_views", "out += d / float(cam.pixels) / n_views"),
    ("imp_P", OI, "imp += i / float(cam.pixels) / n_views", "imp += i / n_views"),
    ("dmse_N", OI, "out += d / (3.0 * cam.pixels) / n_views", "out += d / (3.0 * cam.pixels)"),
    ("g_clamp", GR, "xc = torch.clamp(txz, -lim_x, lim_x) * tz", "xc = txz * tz"),
    ("g_sh_sign", GR, "-c1 * y, c1 * z, -c1 * x,", "c1 * y, c1 * z, -c1 * x,"),
    ("g_sh_c3", GR, "c3d * z * (2 * zz - 3 * xx - 3 * yy)", "c3d * z * (2 * zz - xx - yy)"),
    ("g_cross", GR, "2.0 * pr[\"cb\"][k_t] * dx * dy", "pr[\"cb\"][k_t] * dx * dy"),
    ("g_lowpass", GR, "c = cov[:, 1, 1] + cfg.lowpass", "c = cov[:, 1, 1]"),
    ("g_T_incl", GR, "Tv = torch.exp(excl - start[seg])", "Tv = torch.exp(cs - start[seg])"),
    ("g_relu", GR, "rgb = torch.relu(torch.einsum(\"icn,ni->nc\", p[\"sh\"], Y) + 0.5)", "rgb = torch.einsum(\"icn,ni->nc\", p[\"sh\"], Y) + 0.5"),
    ("g_campos", GR, "campos = -(Wr.T @ tw)\n    d = mu - campos", "campos = -(Wr @ tw)\n    d = mu - campos"),
    ("g_qnorm", GR, "q = p[\"quats\"] / torch.linalg.norm(p[\"quats\"], dim=0, keepdim=True)", "q = p[\"quats\"]"),
    ("g_amax", GR, "alpha = torch.clamp(o[k_t] * torch.exp(power), max=float(cfg.alpha_max))", "alpha = o[k_t] * torch.exp(power)"),
    ("adam_v", AD, "v += (1.0 - b2) * g * g", "v += (1.0 - b2) * abs(g)"),
    # the gradient magnitude bound
    ("gm_suffix_sign", GR, "(Tv[:, None] * rgb_e + s_after / (1.0 - alpha)[:, None])",
     "(Tv[:, None] * rgb_e - s_after / (1.0 - alpha)[:, None])"),
    ("gm_suffix_drop", GR, "s_after / (1.0 - alpha)[:, None])", "0.0 * s_after)"),
    ("gm_colour_T", GR, "gabs[:, ch] * Tv * alpha", "gabs[:, ch] * alpha"),
    ("gm_jac_abs", GR, "r += g.abs() * b_out[:, c:c + 1]", "r += g * b_out[:, c:c + 1]"),
    ("gm_centre_cross", GR, "am * ((ca * dx).abs() + (cb * dy).abs())", "am * (ca * dx).abs()"),
    ("gm_opacity_G", GR, "Mag * G_e * free", "Mag * free"),
    ("gm_resid_abs", GR, "gabs = gc.abs()[:, pix_t].T", "gabs = gc[:, pix_t].T"),
    # pixel masks of the gradient oracle
    ("g_mask_loss", GR, "term = term * torch.from_numpy(np.asarray(mask, np.float64).reshape(cam.height, cam.width))",
     "term = term"),
    ("g_mask_lists", GR, "keep = np.asarray(mask, bool).reshape(-1)[pix]", "keep = np.ones(pix.size, bool)"),
]


def run(name, path, old, new):
    tests = PY_TESTS.get(path, TESTS)
    full = os.path.join(ROOT, path)
    src = open(full).read()
    if src.count(old) != 1:
        return f"{name}: pattern found {src.count(old)} times"
    try:
        open(full, "w").write(src.replace(old, new))
        r = subprocess.run([sys.executable, "-m", "pytest", *tests, "-q", "-x", "-p", "no:cacheprovider"],
                           cwd=ROOT, capture_output=True, text=True, timeout=900)
        tail = [l for l in r.stdout.splitlines() if l.startswith("FAILED") or " passed" in l or " failed" in l]
        verdict = "CAUGHT" if r.returncode != 0 else "MISSED"
        return f"{name}: {verdict}  {tail[0] if tail else r.stdout[-200:]}"
    finally:
        open(full, "w").write(src)


if __name__ == "__main__":
    dirty = subprocess.run(["git", "status", "--porcelain", "--", "oracle"], cwd=ROOT, capture_output=True, text=True)
    if dirty.returncode != 0 or dirty.stdout.strip():
        sys.exit("oracle/ has uncommitted changes (or this is not a git checkout): not planting mistakes")
    want = set(sys.argv[1:])
    for m in MUT:
        if want and m[0] not in want:
            continue
        print(run(*m), flush=True)
    subprocess.run([sys.executable, "-c", "import oracle; oracle.build(force=True)"], cwd=ROOT, check=True)
